"""Index sets of one block round of the stage-1 ordering, written out for the
tests independently of the library: blocks of 16 indices, the circle method
on the N/16 blocks (slot 0 pairs blocks (R, nb-1), slot i pairs blocks
(R+i, R-i) mod nb-1), and block pair q covering its lower block's 16 indices
then its upper block's."""
import numpy as np


def block_sets(N, R):
    nb = N // 16
    sets = []
    for i in range(nb // 2):
        if i == 0:
            x, y = R, nb - 1
        else:
            x, y = (R + i) % (nb - 1), (R - i) % (nb - 1)
        lo, hi = min(x, y), max(x, y)
        sets.append(np.r_[np.arange(16 * lo, 16 * lo + 16), np.arange(16 * hi, 16 * hi + 16)])
    return sets
