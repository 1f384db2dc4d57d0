"""GPU parity: the CUDA path through the C ABI against the CPU oracle on the
same seeded inputs, stage by stage and end to end, plus edge cases.

Tolerances (u = 2^-53, n the size, ||A|| the 2-norm):
  * eigenvalues: |W_gpu - W_oracle| <= 1e-12 ||A|| (the accuracy target) and
    against the constructed spectrum;
  * backward error ||A - Q W Q^T||_F / ||A||_F <= 4 n u and ||Q^T Q - I||_F <= 4 n u;
  * stage-wise products (same inputs): within 10 n u (x ||A||), a bound on
    the difference of two FP64 dot-product summation orders;
  * eigenvectors are compared through residuals/orthogonality or, for
    well-separated spectra, column by column after fixing signs.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2509_00495_gb300 import inputs  # noqa: E402
from block_sets import block_sets  # noqa: E402

U = 2.0 ** -53
UL = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_00495_gb300 import build
    build.build()


def mpj():
    from paper_2509_00495_gb300 import mpj as m
    return m


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def triple(A, W, Q):
    n = A.shape[0]
    be = np.linalg.norm(A - (Q * W) @ Q.T) / np.linalg.norm(A)
    orF = np.linalg.norm(Q.T @ Q - np.eye(n))
    return be / (n * U), orF / (n * U)


def align_signs(Q, R):
    s = np.sign(np.sum(Q * R, axis=0))
    s[s == 0] = 1
    return Q * s


# ---------------------------------------------------------------- DMMA GEMM
@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (64, 64, 64), (70, 33, 129), (130, 200, 17), (5, 300, 257)])
@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
def test_dgemm_matches_numpy(m, n, k, ta, tb):
    rng = np.random.default_rng(m * 7 + n * 3 + k)
    A = rng.standard_normal((k, m) if ta == "T" else (m, k))
    B = rng.standard_normal((n, k) if tb == "T" else (k, n))
    C0 = rng.standard_normal((m, n))
    opA = A.T if ta == "T" else A
    opB = B.T if tb == "T" else B
    got = host(mpj().dgemm(ta, tb, 0.75, dev(A), dev(B), -1.5, dev(C0)))
    ref = 0.75 * opA @ opB - 1.5 * C0
    bound = 2 * (k + 2) * U * (0.75 * np.abs(opA) @ np.abs(opB) + 1.5 * np.abs(C0))
    assert np.all(np.abs(got - ref) <= bound)


# ---------------------------------------------------------------- stage-wise
@pytest.mark.parametrize("n", [50, 97, 130])
def test_newton_schulz_vs_oracle_same_input(n):
    A, lam = inputs.geo_matrix(n, 1e4, seed=n)
    Ql, _, _ = oracle.stage1(A, ordering32=oracle.BLOCK_ROUND_ROBIN)
    ref = oracle.newton_schulz(Ql)
    got = host(mpj().newton_schulz(dev(Ql), 2))
    assert np.abs(got - ref).max() <= 10 * n * U
    assert np.linalg.norm(got.T @ got - np.eye(n), 2) <= n * U


@pytest.mark.parametrize("n", [50, 97, 130])
def test_precondition_vs_oracle_same_input(n):
    A, lam = inputs.geo_matrix(n, 1e4, seed=n + 1)
    Ql, _, _ = oracle.stage1(A, ordering32=oracle.BLOCK_ROUND_ROBIN)
    Qd = oracle.newton_schulz(Ql)
    ref = oracle.precondition(A, Qd)
    got = host(mpj().precondition(dev(A), dev(Qd)))
    assert np.array_equal(got, got.T)
    assert np.abs(got - ref).max() <= 10 * n * U * np.linalg.norm(A, 2)


@pytest.mark.parametrize("n", [2, 3, 33, 64, 97, 130])
def test_jacobi64_round_robin_vs_oracle(n):
    A, lam = inputs.geo_matrix(n, 1e3, seed=3 * n)
    Ql, _, _ = oracle.stage1(A, ordering32=oracle.BLOCK_ROUND_ROBIN)
    Ac = oracle.precondition(A, oracle.newton_schulz(Ql))
    Ac = (Ac + Ac.T) / 2
    tol = n * U * np.linalg.norm(A)
    a_ref, v_ref, sw_ref, _, _, _ = oracle.jacobi(Ac, ordering=oracle.ROUND_ROBIN, tol=tol)
    a, v, sw, off, st = mpj().jacobi64(dev(Ac), tol=tol, ordering="round_robin")
    a, v = host(a), host(v)
    assert st == 0 and off <= tol
    assert abs(sw - sw_ref) <= 1
    nA = np.linalg.norm(A, 2)
    w, w_ref = np.diag(a), np.diag(a_ref)
    assert np.abs(np.sort(w) - np.sort(w_ref)).max() <= 1e-13 * nA
    # same rotation sequence: same pairing of eigenvalues to columns, vectors equal up to sign
    assert np.abs(w - w_ref).max() <= 1e-12 * nA
    assert np.abs(align_signs(v, v_ref) - v_ref).max() <= 1e-9
    assert np.linalg.norm(Ac @ v - v * w) <= 4 * n * U * nA
    assert np.array_equal(a, a.T)


@pytest.mark.parametrize("n", [5, 20, 33, 64])
def test_jacobi64_cyclic_vs_oracle(n):
    A = inputs.randn_sym(n, seed=n)
    tol = n * U * np.linalg.norm(A)
    a_ref, v_ref, sw_ref, _, _, _ = oracle.jacobi(A, ordering=oracle.CYCLIC, tol=tol)
    a, v, sw, off, st = mpj().jacobi64(dev(A), tol=tol, ordering="cyclic")
    a, v = host(a), host(v)
    assert st == 0 and sw == sw_ref
    nA = np.linalg.norm(A, 2)
    assert np.abs(np.diag(a) - np.diag(a_ref)).max() <= 1e-13 * nA
    assert np.abs(align_signs(v, v_ref) - v_ref).max() <= 1e-10


@pytest.mark.parametrize("n", [40, 96, 130])
def test_stage1_vs_oracle_block_ordering(n):
    A, lam = inputs.geo_matrix(n, 1e3, seed=5 * n)
    Ql_ref, A32_ref, info = oracle.stage1(A, ordering32=oracle.BLOCK_ROUND_ROBIN)
    Ql, sw, off32 = mpj().stage1(dev(A))
    Ql = host(Ql)
    nA = np.linalg.norm(A)
    assert abs(sw - info.sweeps32) <= 1
    assert off32 <= n * UL * nA
    assert np.linalg.norm(Ql.T @ Ql - np.eye(n), 2) <= 8 * n * UL
    D = np.diag(Ql.T @ A @ Ql)
    assert np.linalg.norm(A @ Ql - Ql * D, 2) <= 8 * n * UL * np.linalg.norm(A, 2)
    # same ordering: the FP32 eigenvalue approximations agree with the oracle's to the FP32 level
    D_ref = np.diag(Ql_ref.T @ A @ Ql_ref)
    assert np.abs(np.sort(D) - np.sort(D_ref)).max() <= 8 * n * UL * np.linalg.norm(A, 2)


# ---------------------------------------------------------------- end to end
@pytest.mark.parametrize("n", [1, 2, 3, 17, 96, 130, 257])
def test_syev_mixed_vs_oracle(n):
    A, lam = inputs.geo_matrix(n, 1e3, seed=11 * n) if n > 1 else (np.array([[-0.7]]), np.array([-0.7]))
    r = mpj().syev_ex(dev(A), ordering="round_robin")
    W, Q = host(r.W), host(r.Q)
    Wr, Qr, info = oracle.syev_mixed(A, ordering32=oracle.BLOCK_ROUND_ROBIN, ordering64=oracle.ROUND_ROBIN,
                                     threshold=True)
    nA = np.linalg.norm(A, 2)
    assert r.status == 0
    assert np.all(np.diff(W) >= 0)
    assert np.abs(W - Wr).max() <= 1e-12 * nA
    assert np.abs(W - np.sort(lam)).max() <= 1e-12 * nA
    be, orF = triple(A, W, Q)
    assert be <= 4 and orF <= 4, (be, orF)
    assert abs(r.info["sweeps64"] - info.sweeps64) <= 1
    assert r.info["sweeps64"] < 10  # the paper's "fewer than 10 sweeps"


@pytest.mark.parametrize("n", [33, 96])
def test_syev_plain_vs_oracle(n):
    A, lam = inputs.geo_matrix(n, 1e3, seed=13 * n)
    r = mpj().syev_ex(dev(A), method="plain", ordering="round_robin")
    W, Q = host(r.W), host(r.Q)
    Wr, Qr, info = oracle.syev_plain(A, ordering64=oracle.ROUND_ROBIN, threshold=True)
    nA = np.linalg.norm(A, 2)
    assert np.abs(W - Wr).max() <= 1e-12 * nA
    assert abs(r.info["sweeps64"] - info.sweeps64) <= 1
    be, orF = triple(A, W, Q)
    assert be <= 4 and orF <= 8


def test_syev_cyclic_fp64_stage_vs_oracle():
    n = 64
    A, lam = inputs.geo_matrix(n, 1e3, seed=21)
    r = mpj().syev_ex(dev(A), ordering="cyclic")
    Wr, Qr, info = oracle.syev_mixed(A, ordering32=oracle.BLOCK_ROUND_ROBIN, ordering64=oracle.CYCLIC)
    assert abs(r.info["sweeps64"] - info.sweeps64) <= 1
    assert np.abs(host(r.W) - Wr).max() <= 1e-12 * np.linalg.norm(A, 2)


@pytest.mark.parametrize("threshold", [0, 1])
def test_threshold_option_vs_oracle(threshold):
    """The threshold variant (skip |a_pq| <= tol/n) on and off, against the oracle
    with the same rule: same sweeps (+-1), same eigenvalues, same accuracy."""
    n = 130
    A, lam = inputs.geo_matrix(n, 1e6, seed=5)
    r = mpj().syev_ex(dev(A), threshold=threshold, ordering="round_robin")
    Wr, _, info = oracle.syev_mixed(A, ordering32=oracle.BLOCK_ROUND_ROBIN, ordering64=oracle.ROUND_ROBIN,
                                    threshold=bool(threshold))
    assert abs(r.info["sweeps64"] - info.sweeps64) <= 1
    assert np.abs(host(r.W) - Wr).max() <= 1e-12 * np.linalg.norm(A, 2)
    be, orF = triple(A, host(r.W), host(r.Q))
    assert be <= 4 and orF <= 4


def test_paper_sweep_claims_small_cases():
    """Sec. 5.2.3: about 2 FP64 sweeps for arithmetic spectra, up to 4 for geometric ones."""
    A, _ = inputs.ari_matrix(200, 500, seed=1)
    assert mpj().syev_ex(dev(A)).info["sweeps64"] <= 3
    A, _ = inputs.geo_matrix(200, 500, seed=1)
    assert mpj().syev_ex(dev(A)).info["sweeps64"] <= 5


# ---------------------------------------------------------------- edge cases
def test_diagonal_input_needs_no_sweep():
    d = np.array([3.0, -1.0, 2.0, 0.5, -7.0])
    r = mpj().syev_ex(dev(np.diag(d)))
    assert r.info["sweeps64"] == 0
    assert np.array_equal(host(r.W), np.sort(d))
    Q = host(r.Q)
    assert np.array_equal(np.abs(Q), np.abs(Q).round())  # a signed permutation


def test_nonfinite_input_is_rejected():
    A = inputs.randn_sym(10, 1)
    A[3, 4] = A[4, 3] = np.nan
    with pytest.raises(mpj().MPJError) as e:
        mpj().syev_ex(dev(A))
    assert e.value.status == mpj().MPJ_ENONFINITE


def test_symmetry_check():
    A = inputs.randn_sym(10, 2)
    A[1, 2] += 1e-3
    with pytest.raises(mpj().MPJError) as e:
        mpj().syev_ex(dev(A), check_symmetry=1)
    assert e.value.status == mpj().MPJ_ENOTSYM


def test_sweep_cap_reports_not_converged():
    A = inputs.randn_sym(40, 3)
    r = mpj().syev_ex(dev(A), method="plain", max_sweeps64=1)
    assert r.status == mpj().MPJ_NOT_CONVERGED and r.info["sweeps64"] == 1
    assert r.info["off_final"] > r.info["tol"]


def test_caller_workspace():
    m = mpj()
    A, lam = inputs.geo_matrix(70, 1e2, seed=8)
    nbytes = m.syev_workspace(70)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    r = m.syev_ex(dev(A), workspace=ws)
    assert np.abs(host(r.W) - np.sort(lam)).max() <= 1e-12
    small = torch.empty(nbytes // 2, dtype=torch.uint8, device="cuda")
    with pytest.raises(m.MPJError) as e:
        m.syev_ex(dev(A), workspace=small)
    assert e.value.status == m.MPJ_EWORKSPACE


def test_bitwise_deterministic():
    A, _ = inputs.geo_matrix(150, 1e4, seed=4)
    r1 = mpj().syev_ex(dev(A))
    r2 = mpj().syev_ex(dev(A))
    assert torch.equal(r1.W, r2.W) and torch.equal(r1.Q, r2.Q)


def test_polish_option_keeps_accuracy():
    A, lam = inputs.geo_matrix(120, 1e5, seed=6)
    r = mpj().syev_ex(dev(A), polish=1)
    be, orF = triple(A, host(r.W), host(r.Q))
    assert be <= 4 and orF <= 4


# ---------------------------------------------------------------- full sizes (properties)
def _gpu_triple(A_t, W_t, Q_t):
    n = A_t.shape[0]
    be = torch.linalg.norm(A_t - (Q_t * W_t) @ Q_t.T) / torch.linalg.norm(A_t)
    orF = torch.linalg.norm(Q_t.T @ Q_t - torch.eye(n, dtype=torch.float64, device="cuda"))
    return be.item() / (n * U), orF.item() / (n * U)


def test_clustered_1024_properties():
    A, lam = inputs.clustered_1024(seed=0)
    A_t = dev(A)
    r = mpj().syev_ex(A_t)
    W = host(r.W)
    assert np.abs(W - np.sort(lam)).max() <= 1e-12 * np.abs(lam).max()
    be, orF = _gpu_triple(A_t, r.W, r.Q)
    assert be <= 4 and orF <= 4, (be, orF)
    # the 32-eigenvalue cluster near 0.5: individual vectors are unpinned, the subspace is
    rng = np.random.default_rng(0)
    Qtrue = inputs.haar_orthogonal(1024, rng)
    cl = np.arange(992, 1024)
    order = np.argsort(lam)
    pos = np.searchsorted(np.sort(lam), lam[cl])
    Qc = host(r.Q)[:, pos]
    s = np.linalg.svd(Qtrue[:, cl].T @ Qc, compute_uv=False)
    assert s.min() >= 1 - 1e-9
    assert r.info["sweeps64"] < 30


def test_geo_4096_properties():
    A, lam = inputs.geo_4096(seed=0)
    A_t = dev(A)
    r = mpj().syev_ex(A_t)
    assert r.status == 0
    W = host(r.W)
    assert np.abs(W - np.sort(lam)).max() <= 1e-12
    be, orF = _gpu_triple(A_t, r.W, r.Q)
    assert be <= 4 and orF <= 4, (be, orF)


# ---------------------------------------------------------------- batched
def test_batched_vs_oracle_sample():
    rng = np.random.default_rng(5)
    sizes = [1, 2, 8, 9, 31, 64, 100, 129, 200, 256]
    mats = []
    for n in sizes:
        g = rng.standard_normal((n, n)) / np.sqrt(n)
        mats.append((g + g.T) / 2)
    Ws, Qs, sweeps, st = mpj().syev_batched([dev(a) for a in mats])
    assert st == 0
    for a, W, Q, sw in zip(mats, Ws, Qs, sweeps):
        n = a.shape[0]
        W, Q = host(W), host(Q)
        Wr, Qr, info = oracle.syev_mixed(a, ordering32=oracle.ROUND_ROBIN, ordering64=oracle.ROUND_ROBIN,
                                         threshold=True)
        nA = max(np.linalg.norm(a, 2), 1e-300)
        assert np.abs(W - Wr).max() <= 1e-12 * nA
        be, orF = triple(a, W, Q)
        assert be <= 4 and orF <= 4, (n, be, orF)
        assert abs(sw - info.sweeps64) <= 1


# ---------------------------------------------------------------- backward
def test_backward_vs_oracle_and_closed_forms():
    rng = np.random.default_rng(3)
    n, b = 40, 3
    Ws, Qs, dWs, dQs = [], [], [], []
    for i in range(b):
        lam = inputs.gapped_spectrum(n, rng, gap=1e-3)
        A = inputs.from_spectrum(lam, inputs.haar_orthogonal(n, rng))
        r = mpj().syev_ex(dev(A))
        Ws.append(r.W)
        Qs.append(r.Q)
        dWs.append(dev(rng.standard_normal(n)))
        dQs.append(dev(rng.standard_normal((n, n))))
    W, Q, dW, dQ = torch.stack(Ws), torch.stack(Qs), torch.stack(dWs), torch.stack(dQs)
    dA = host(mpj().syev_backward(W, Q, dW, dQ))
    for i in range(b):
        ref = oracle.eigh_backward(host(W[i]), host(Q[i]), host(dW[i]), host(dQ[i]))
        assert np.abs(dA[i] - ref).max() <= 1e-10 * np.abs(ref).max()
        assert np.array_equal(dA[i], dA[i].T)
    dA0 = host(mpj().syev_backward(W[0], Q[0], dW[0], None))
    Qh = host(Q[0])
    assert np.abs(dA0 - Qh @ np.diag(host(dW[0])) @ Qh.T).max() <= 1e-13


def test_backward_degenerate_is_reported():
    m = mpj()
    W = dev(np.array([1.0, 1.0, 2.0]))
    Q = dev(np.eye(3))
    with pytest.raises(m.MPJError) as e:
        m.syev_backward(W, Q, None, dev(np.ones((3, 3))))
    assert e.value.status == m.MPJ_EDEGENERATE


def test_autograd_matches_central_differences():
    n = 12
    rng = np.random.default_rng(9)
    lam = inputs.gapped_spectrum(n, rng, gap=0.05)
    A0 = inputs.from_spectrum(lam, inputs.haar_orthogonal(n, rng))
    dW = dev(rng.standard_normal(n))
    dQ = dev(rng.standard_normal((n, n)))
    A = dev(A0).requires_grad_(True)
    W, Q = mpj().eigh(A)
    Qref = Q.detach().clone()
    (W * dW).sum().backward(retain_graph=True)
    gW = A.grad.clone()
    A.grad = None
    (Q * dQ).sum().backward()
    g = gW + A.grad

    def loss(M):
        w, q = mpj().eigh(M)
        s = torch.sign((q * Qref).sum(0))
        return ((w * dW).sum() + (q * s * dQ).sum()).item()

    h = 1e-6
    for (i, j) in [(0, 0), (2, 5), (7, 1), (11, 11)]:
        E = torch.zeros(n, n, dtype=torch.float64, device="cuda")
        E[i, j] += 0.5
        E[j, i] += 0.5
        fd = (loss(A.detach() + h * E) - loss(A.detach() - h * E)) / (2 * h)
        an = (g * E).sum().item()
        assert fd == pytest.approx(an, rel=1e-6, abs=1e-7)


# ---------------------------------------------------------------- second preconditioning pass (option)
@pytest.mark.parametrize("n", [96, 257])
def test_two_pass_preconditioning_vs_oracle(n):
    A, lam = inputs.geo_matrix(n, 1e6, seed=17 * n)
    r1 = mpj().syev_ex(dev(A), ordering="round_robin")
    r2 = mpj().syev_ex(dev(A), precond_passes=2, ordering="round_robin")
    W, Q = host(r2.W), host(r2.Q)
    Wr, _, _ = oracle.syev_mixed(A, ordering32=oracle.BLOCK_ROUND_ROBIN, ordering64=oracle.ROUND_ROBIN)
    nA = np.linalg.norm(A, 2)
    assert r2.status == 0 and r2.info["sweeps32_pass2"] >= 1
    assert np.abs(W - Wr).max() <= 1e-12 * nA
    assert np.abs(W - np.sort(lam)).max() <= 1e-12 * nA
    be, orF = triple(A, W, Q)
    assert be <= 4 and orF <= 4, (be, orF)
    assert r2.info["sweeps64"] <= r1.info["sweeps64"]


def test_two_pass_geo_4096_properties():
    A, lam = inputs.geo_4096(seed=0)
    A_t = dev(A)
    r = mpj().syev_ex(A_t, precond_passes=2)
    assert r.status == 0
    assert np.abs(host(r.W) - np.sort(lam)).max() <= 1e-12
    be, orF = _gpu_triple(A_t, r.W, r.Q)
    assert be <= 4 and orF <= 4, (be, orF)


@pytest.mark.parametrize("group", ["256", "512", "1024"])
def test_batched_each_group_size(group, monkeypatch):
    """Every thread-group size the autotuner can pick gives oracle-exact results."""
    monkeypatch.setenv("MPJ_BATCHED_GROUP", group)
    rng = np.random.default_rng(int(group))
    sizes = [3, 17, 64, 130, 256, 40 + int(group) // 256]  # a distinct size list -> a fresh plan
    mats = []
    for n in sizes:
        g = rng.standard_normal((n, n)) / np.sqrt(n)
        mats.append((g + g.T) / 2)
    Ws, Qs, sweeps, st = mpj().syev_batched([dev(a) for a in mats])
    assert st == 0
    for a, W, Q in zip(mats, Ws, Qs):
        W, Q = host(W), host(Q)
        Wr, _, _ = oracle.syev_mixed(a, ordering32=oracle.ROUND_ROBIN, ordering64=oracle.ROUND_ROBIN)
        assert np.abs(W - Wr).max() <= 1e-12 * max(np.linalg.norm(a, 2), 1e-300)
        be, orF = triple(a, W, Q)
        assert be <= 4 and orF <= 4


def test_batched_graph_replay_and_autotune():
    """Repeated solves on fixed buffers replay the planned graph; new data, same plan."""
    m = mpj()
    rng = np.random.default_rng(77)
    sizes = list(rng.integers(8, 257, size=24))
    solver = m.BatchedSolver(sizes)
    for trial in range(3):
        mats = []
        for n in sizes:
            g = rng.standard_normal((n, n)) / np.sqrt(n)
            mats.append((g + g.T) / 2)
        Ws, Qs, sweeps, st = solver.solve([dev(a) for a in mats])
        assert st == 0
        for a, W, Q in zip(mats, Ws, Qs):
            wr = np.linalg.eigvalsh(a)
            assert np.abs(host(W) - wr).max() <= 1e-12 * np.linalg.norm(a, 2)
            be, orF = triple(a, host(W), host(Q))
            assert be <= 4 and orF <= 4
    assert solver.group_size() in (0, 256, 512, 1024)


def test_batched_rejects_nonfinite():
    m = mpj()
    a = np.eye(5)
    a[1, 2] = a[2, 1] = np.inf
    with pytest.raises(m.MPJError) as e:
        m.syev_batched([dev(a), dev(np.eye(3))])
    assert e.value.status == m.MPJ_ENONFINITE


# ---------------------------------------------------------------- stage-1 tensor-core block product
@pytest.mark.gpu
@pytest.mark.parametrize("N,R", [(64, 0), (96, 3), (320, 7), (1024, 30)])
def test_stage1_panel_tensor_cores(N, R):
    """3xTF32 tcgen05 block product vs an FP64 numpy product of the same FP32 data."""
    rng = np.random.default_rng(N + R)
    X = rng.standard_normal((N, N)).astype(np.float32)          # logical matrix
    Uq = np.stack([np.linalg.qr(rng.standard_normal((32, 32)))[0] for _ in range(N // 32)]).astype(np.float32)
    Xd = torch.from_numpy(np.ascontiguousarray(X.T)).cuda()       # column-major storage
    Ud = torch.from_numpy(np.ascontiguousarray(Uq.transpose(0, 2, 1))).cuda()
    sets = block_sets(N, R)
    ref = np.zeros((N, N))
    for q, I in enumerate(sets):
        ref[:, I] = X[:, I].astype(np.float64) @ Uq[q].astype(np.float64)
    out = mpj().stage1_panel(R, Ud, Xd).cpu().numpy().T
    scale = np.abs(X).max() * np.sqrt(32)
    assert np.abs(out - ref).max() <= 2.0 ** -19 * scale
    outT = mpj().stage1_panel(R, Ud, Xd, transpose_out=True).cpu().numpy().T
    assert np.abs(outT - ref.T).max() <= 2.0 ** -19 * scale


@pytest.mark.gpu
def test_stage1_panel_timeout_is_reported():
    """Failure detection without a fault: with no tensor-core work issued, the
    kernel's bounded completion wait runs out, MPJ_ETIMEOUT comes back, the
    output is untouched and the next call works."""
    m = mpj()
    N = 64
    rng = np.random.default_rng(0)
    X = torch.from_numpy(rng.standard_normal((N, N)).astype(np.float32)).cuda()
    U = torch.from_numpy(np.stack([np.eye(32, dtype=np.float32)] * (N // 32))).cuda()
    with pytest.raises(RuntimeError, match="MPJ_ETIMEOUT"):
        m.stage1_panel(0, U, X, _test_no_commit=True)
    out = m.stage1_panel(0, U, X)  # identity factors: the product is X itself
    torch.cuda.synchronize()
    assert torch.allclose(out, X, rtol=2.0 ** -19, atol=0)


_OVERLAP_SCRIPT = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_2509_00495_gb300 import inputs, mpj
A, lam = inputs.geo_matrix(300, 1e4, seed=7)
r = mpj.syev_ex(torch.from_numpy(A).cuda())
torch.cuda.synchronize()
np.save(sys.argv[2], np.concatenate([r.W.cpu().numpy()[None, :], r.Q.cpu().numpy()]))
"""


@pytest.mark.gpu
def test_side_stream_overlap_is_bitwise_neutral(tmp_path):
    """The V updates of stage 1 and of the FP64 sweeps give the same bits on
    the private side stream as on the caller's stream (n = 300 >= 256 turns
    the overlap on in both); a difference would flag a race between the
    rotation rounds and the V updates."""
    import os
    import subprocess
    import sys as _sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = tmp_path / "run.py"
    script.write_text(_OVERLAP_SCRIPT)
    outs = []
    for flag in ("1", "0"):
        out = tmp_path / f"wq{flag}.npy"
        env = dict(os.environ, MPJ_JACOBI_OVERLAP=flag)
        subprocess.run([_sys.executable, str(script), root, str(out)], check=True, env=env, timeout=300)
        outs.append(np.load(out))
    assert np.array_equal(outs[0], outs[1])


_GRAPH_SCRIPT = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_2509_00495_gb300 import inputs, mpj
outs, wss = [], {}
# sizes and workspaces in turn (each workspace kept alive, so each has its own
# address): cache hits, misses, and more keys than the cache holds
# (evictions); the same size again with another workspace
for n, ws_id in ((300, 0), (520, 1), (300, 0), (300, 2), (700, 3), (420, 4), (520, 1), (300, 0)):
    A, lam = inputs.geo_matrix(n, 1e4, seed=n + ws_id)
    if ws_id not in wss:
        wss[ws_id] = torch.empty(mpj.syev_workspace(n), dtype=torch.uint8, device="cuda")
    ws = wss[ws_id]
    r = mpj.syev_ex(torch.from_numpy(A).cuda(), workspace=ws)
    torch.cuda.synchronize()
    assert r.status == 0
    outs.append(np.concatenate([r.W.cpu().numpy(), r.Q.cpu().numpy().ravel()]))
np.save(sys.argv[2], np.concatenate(outs))
"""


@pytest.mark.gpu
def test_stage1_sweep_graphs_are_bitwise_neutral(tmp_path):
    """Stage-1 sweeps replayed from the per-workspace CUDA-graph cache give the
    same bits as the same sweeps enqueued kernel by kernel
    (MPJ_STAGE1_GRAPH=0), over a sequence of sizes and workspaces that hits,
    misses and evicts cache entries."""
    import os
    import subprocess
    import sys as _sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = tmp_path / "run.py"
    script.write_text(_GRAPH_SCRIPT)
    outs = []
    for flag in ("1", "0"):
        out = tmp_path / f"g{flag}.npy"
        env = dict(os.environ, MPJ_STAGE1_GRAPH=flag)
        subprocess.run([_sys.executable, str(script), root, str(out)], check=True, env=env, timeout=300)
        outs.append(np.load(out))
    assert np.array_equal(outs[0], outs[1])


_STAGE1_TC_SCRIPT = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_2509_00495_gb300 import inputs, mpj
A, lam = inputs.geo_matrix(300, 1e4, seed=17)
r = mpj.syev_ex(torch.from_numpy(A).cuda())
torch.cuda.synchronize()
np.save(sys.argv[2], np.concatenate([r.W.cpu().numpy()[None, :], r.Q.cpu().numpy()]))
print(r.status, r.info["sweeps32"], r.info["sweeps64"])
"""


@pytest.mark.gpu
def test_stage1_tensor_core_option_solve(tmp_path):
    """The whole mixed solve with the stage-1 A update on the tcgen05 panel
    (MPJ_STAGE1_TC=1: U column-major for the panel, the V update on the FP32
    pipe reading the same layout) reaches the FP64 accuracy bounds and the
    known spectrum, like the default FP32-pipe stage."""
    import os
    import subprocess
    import sys as _sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = tmp_path / "run.py"
    script.write_text(_STAGE1_TC_SCRIPT)
    out = tmp_path / "wq.npy"
    env = dict(os.environ, MPJ_STAGE1_TC="1")
    res = subprocess.run([_sys.executable, str(script), root, str(out)], check=True, env=env, timeout=300,
                         capture_output=True, text=True)
    status, sw32, sw64 = (int(x) for x in res.stdout.split()[-3:])
    assert status == 0 and sw32 >= 1
    WQ = np.load(out)
    W, Q = WQ[0], WQ[1:]
    A, lam = inputs.geo_matrix(300, 1e4, seed=17)
    nA = np.linalg.norm(A, 2)
    assert np.abs(W - np.sort(lam)).max() <= 1e-12 * nA
    be, orF = triple(A, W, Q)
    assert be <= 4 and orF <= 8, (be, orF)
    assert sw64 < 10


@pytest.mark.gpu
@pytest.mark.parametrize("m,n,k,ta,tb", [(64, 64, 64, "N", "N"), (130, 70, 300, "N", "N"), (200, 129, 513, "T", "N"),
                                         (96, 200, 256, "N", "T"), (257, 65, 1000, "T", "T")])
def test_dgemm_tc_matches_numpy(m, n, k, ta, tb):
    """The tensor-core FP64 product (exact bf16 slices) within the FP64 product's
    componentwise error bound, on tiles, ragged edges and every transpose."""
    rng = np.random.default_rng(m * 5 + n * 11 + k)
    A = rng.standard_normal((k, m) if ta == "T" else (m, k))
    B = rng.standard_normal((n, k) if tb == "T" else (k, n))
    C0 = rng.standard_normal((m, n))
    opA = A.T if ta == "T" else A
    opB = B.T if tb == "T" else B
    got = host(mpj().dgemm_tc(ta, tb, 0.75, dev(A), dev(B), -1.5, dev(C0)))
    ref = 0.75 * opA @ opB - 1.5 * C0
    bound = 2 * (k + 2) * U * (0.75 * np.abs(opA) @ np.abs(opB) + 1.5 * np.abs(C0))
    assert np.all(np.abs(got - ref) <= bound)
    # and much closer than the bound: an exact-slice product errs by a few units
    # of the output's last place, not by k of them
    assert np.abs(got - ref).max() <= 64 * U * (np.abs(opA) @ np.abs(opB)).max()


_ENGINE_SCRIPT = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_2509_00495_gb300 import inputs, mpj
A, lam = inputs.geo_matrix(300, 1e6, seed=11)
r = mpj.syev_ex(torch.from_numpy(A).cuda())
torch.cuda.synchronize()
assert r.status == 0
np.save(sys.argv[2], np.concatenate([r.W.cpu().numpy()[None, :], r.Q.cpu().numpy()]))
"""


@pytest.mark.gpu
def test_gemm_engines_agree(tmp_path):
    """The FP64 products on the tensor cores (default) and on the DMMA kernel
    (MPJ_GEMM_TC=0) both give an FP64-accurate solve with the same spectrum."""
    import os
    import subprocess
    import sys as _sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = tmp_path / "run.py"
    script.write_text(_ENGINE_SCRIPT)
    A, lam = inputs.geo_matrix(300, 1e6, seed=11)
    res = []
    for flag in ("1", "0"):
        out = tmp_path / f"wq{flag}.npy"
        env = dict(os.environ, MPJ_GEMM_TC=flag)
        subprocess.run([_sys.executable, str(script), root, str(out)], check=True, env=env, timeout=300)
        wq = np.load(out)
        W, Q = wq[0], wq[1:]
        be, orF = triple(A, W, Q)
        assert be <= 4 and orF <= 4, (flag, be, orF)
        res.append(W)
    nA = np.linalg.norm(A, 2)
    assert np.abs(res[0] - res[1]).max() <= 1e-12 * nA
    assert np.abs(res[0] - np.sort(lam)).max() <= 1e-12 * nA
