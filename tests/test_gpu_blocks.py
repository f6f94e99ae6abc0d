"""Block operations through the C ABI: batched complex GEMM and block inverse, FP64 (CUDA cores)
and mixed (tensor cores, exact split-BF16 slices), against numpy complex128."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
negf = pytest.importorskip("paper_1510_04686_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    negf._build.build()
    negf.library()


def _rand(rng, shape, scale=1.0):
    return scale * (rng.normal(size=shape) + 1j * rng.normal(size=shape))


def _op(X, op):
    if op == "N":
        return X
    Xt = np.swapaxes(X, -1, -2)
    return Xt.conj() if op == "C" else Xt


def _bound(A, B, opA, opB):
    """Per-entry scale K * max_k |op(A)_mk| * max_k |op(B)_kn| of the normwise GEMM error."""
    a = np.abs(_op(A, opA))
    b = np.abs(_op(B, opB))
    K = a.shape[-1]
    return K * a.max(axis=-1)[..., :, None] * b.max(axis=-2)[..., None, :]


# M = 300 has an odd number (3) of 128-row tiles, which the CTA-pair kernel pads to an even count;
# K = 1000 is longer than the operand strip the single-read slicing kernel keeps in shared
# memory, so it takes the two-pass slicing kernel
CASES = [(40, 40, 40), (77, 130, 50), (128, 128, 128), (200, 160, 96), (300, 200, 150),
         (400, 400, 400), (64, 48, 1000)]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("M,N,K", CASES)
def test_zgemm_matches_numpy(prec, M, N, K):
    rng = np.random.default_rng(M + 7 * N + 13 * K)
    nb = 3
    for opA, opB in [("N", "N"), ("C", "N"), ("N", "C"), ("T", "T")]:
        A = _rand(rng, (nb,) + ((M, K) if opA == "N" else (K, M)))
        B = _rand(rng, (nb,) + ((K, N) if opB == "N" else (N, K)))
        C0 = _rand(rng, (nb, M, N))
        al, be = 0.7 - 0.2j, -0.4 + 1.1j
        ref = al * (_op(A, opA) @ _op(B, opB)) + be * C0
        C = torch.as_tensor(C0.copy(), device="cuda")
        negf.zgemm(torch.as_tensor(A, device="cuda"), torch.as_tensor(B, device="cuda"), C,
                   alpha=al, beta=be, opA=opA, opB=opB, precision=prec)
        got = C.cpu().numpy()
        tol = (1e-15 if prec == 0 else 1e-13) * abs(al) * _bound(A, B, opA, opB) + 1e-15 * np.abs(C0)
        assert np.all(np.abs(got - ref) <= tol + 1e-300), (opA, opB, np.abs(got - ref).max())


@pytest.mark.parametrize("al,be", [(1.0, 0.0), (-1.0, 1.0), (2.0, -1.0), (-0.3, 0.25),
                                   (0.5j, 1.0), (1.0, 0.6 - 0.8j)])
def test_zgemm_coefficient_forms(al, be):
    """Each form of alpha and beta (zero, one, minus one, real, complex) in the tensor-core
    epilogue gives alpha A B + beta C."""
    rng = np.random.default_rng(int(abs(al) * 100 + abs(be) * 10))
    nb, M, N, K = 2, 150, 140, 130
    A, B, C0 = _rand(rng, (nb, M, K)), _rand(rng, (nb, K, N)), _rand(rng, (nb, M, N))
    ref = al * (A @ B) + be * C0
    C = torch.as_tensor(C0.copy(), device="cuda")
    negf.zgemm(torch.as_tensor(A, device="cuda"), torch.as_tensor(B, device="cuda"), C,
               alpha=al, beta=be, precision=1)
    tol = 1e-13 * abs(al) * _bound(A, B, "N", "N") + 1e-15 * np.abs(C0)
    assert np.all(np.abs(C.cpu().numpy() - ref) <= tol + 1e-300)


@pytest.mark.parametrize("prec", [0, 1])
def test_zgemm_shared_operand_and_dynamic_range(prec):
    rng = np.random.default_rng(3)
    nb, M, N, K = 4, 96, 80, 112
    A = _rand(rng, (nb, M, K))
    # rows and columns spanning 16 orders of magnitude: the per-row / per-column power-of-two
    # scaling must keep each entry's error relative to its own row and column
    A *= (10.0 ** rng.uniform(-8, 8, (nb, M, 1)))
    B = _rand(rng, (K, N)) * (10.0 ** rng.uniform(-8, 8, (1, N)))
    ref = A @ B
    C = negf.zgemm(torch.as_tensor(A, device="cuda"), torch.as_tensor(B, device="cuda"),
                   precision=prec).cpu().numpy()
    tol = 1e-13 * _bound(A, np.broadcast_to(B, (nb, K, N)), "N", "N")
    assert np.all(np.abs(C - ref) <= tol)


def test_zgemm_mixed_is_deterministic():
    rng = np.random.default_rng(9)
    A = torch.as_tensor(_rand(rng, (2, 200, 200)), device="cuda")
    B = torch.as_tensor(_rand(rng, (2, 200, 200)), device="cuda")
    c1 = negf.zgemm(A, B, precision=1).cpu().numpy()
    c2 = negf.zgemm(A, B, precision=1).cpu().numpy()
    assert np.array_equal(c1, c2)


@pytest.mark.parametrize("prec,steps", [(0, 0), (1, 2), (1, 3)])
@pytest.mark.parametrize("n", [40, 130, 400])
def test_zinv_matches_numpy(prec, steps, n):
    rng = np.random.default_rng(n)
    nb = 3
    H = _rand(rng, (nb, n, n), 1.0 / np.sqrt(n))
    H = 0.5 * (H + np.swapaxes(H, 1, 2).conj())
    z = np.array([0.1 + 1e-3j, 0.37 + 1e-6j, -0.9 + 1e-6j])
    M = z[:, None, None] * np.eye(n) - H
    ref = np.linalg.inv(M)
    X, st = negf.zinv(torch.as_tensor(M.copy(), device="cuda"), precision=prec,
                      refine_steps=steps)
    X = X.cpu().numpy()
    assert np.all(st.cpu().numpy() == 0)
    for p in range(nb):
        kappa = np.linalg.norm(M[p], 2) * np.linalg.norm(ref[p], 2)
        err = np.abs(X[p] - ref[p]).max() / np.abs(ref[p]).max()
        assert err < 1e-15 * kappa * n, (p, err, kappa)


@pytest.mark.parametrize("prec,steps", [(0, 0), (1, 2)])
@pytest.mark.parametrize("n", [200, 400])
def test_zinv_large_batch(prec, steps, n):
    """A batch of 100 matrices at the sweep's sizes (panel Gauss-Jordan with batched trailing
    updates, FP64 and FP32 + Newton-Schulz); same accuracy bar as the small batches."""
    rng = np.random.default_rng(n + 1)
    nb = 100
    H = _rand(rng, (nb, n, n), 1.0 / np.sqrt(n))
    H = 0.5 * (H + np.swapaxes(H, 1, 2).conj())
    z = (np.linspace(-1.5, 1.5, nb) + 1j * np.geomspace(1e-6, 1e-2, nb))
    M = z[:, None, None] * np.eye(n) - H
    X, st = negf.zinv(torch.as_tensor(M.copy(), device="cuda"), precision=prec,
                      refine_steps=steps)
    X = X.cpu().numpy()
    assert np.all(st.cpu().numpy() == 0)
    ref = np.linalg.inv(M)
    for p in range(0, nb, 7):
        kappa = np.linalg.norm(M[p], 2) * np.linalg.norm(ref[p], 2)
        err = np.abs(X[p] - ref[p]).max() / np.abs(ref[p]).max()
        assert err < 1e-15 * kappa * n, (p, err, kappa)
    # every item: residual of the inverse
    R = np.einsum("pij,pjk->pik", M, X) - np.eye(n)
    assert np.all(np.isfinite(X)) and np.abs(R).max() < 1e-6


def test_zinv_reports_singular():
    M = torch.zeros((2, 8, 8), dtype=torch.complex128, device="cuda")
    M[0] = torch.eye(8, dtype=torch.complex128, device="cuda")
    X, st = negf.zinv(M, precision=0)
    st = st.cpu().numpy()
    assert st[0] == 0 and (st[1] & 2)


def test_zgemm_every_kernel_configuration():
    """All tensor-core kernel configurations (pipeline depth, K-part policy) give the product to
    the stated accuracy; the default is restored afterwards."""
    rng = np.random.default_rng(21)
    old = negf.tc_config()
    try:
        for nb, n in ((3, 400), (2, 300)):  # 4 and 3 row tiles (one CTA or a CTA pair per MMA)
            A = _rand(rng, (nb, n, n))
            B = _rand(rng, (nb, n, n))
            ref = A @ B
            tol = 1e-13 * _bound(A, B, "N", "N")
            At, Bt = torch.as_tensor(A, device="cuda"), torch.as_tensor(B, device="cuda")
            for c in range(negf.tc_config_count()):
                negf.tc_config(c)
                C = negf.zgemm(At, Bt, precision=1).cpu().numpy()
                assert np.all(np.abs(C - ref) <= tol), (n, c)
    finally:
        negf.tc_config(old)
