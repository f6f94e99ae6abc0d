"""Adjoint RGF (negf_rgf_adjoint) against the oracle's dense gradient and finite differences.

L = sum_p [ sum_j c_pj n_j(p) + sum_i d_pi j_i(p) ],  dL/dV_q = Re[(G^< Om G + G^H Om G^<)_qq]
summed over points (oracle.gradient_dense, pinned to central differences on the CPU).
"""
import numpy as np
import pytest

import oracle as O
from workloads import make_device

torch = pytest.importorskip("torch")
negf = pytest.importorskip("paper_1510_04686_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    negf._build.build()
    negf.library()


def _setup(N, b, seed, n_pts, scatter=False):
    dev = make_device(N, b, seed, ge_frac=0.2)
    rng = np.random.default_rng(seed)
    E = np.linspace(-1.3, 1.1, n_pts)
    V = rng.uniform(-0.2, 0.2, (N, b))
    c = rng.normal(size=(n_pts, N * b))
    d = rng.normal(size=(n_pts, N - 1))
    sR = sL = None
    if scatter:
        gam = 0.03 * rng.random((n_pts, N * b))
        sR = 0.01 * rng.normal(size=(n_pts, N * b)) - 1j * gam
        sL = 1j * 0.5 * 2 * gam
    return dev, E, V, c, d, sR, sL


def _gpu_grad(dev, E, V, c, d, opt, sR=None, sL=None):
    Hd = torch.as_tensor(dev.D[None], device="cuda")
    Hu = torch.as_tensor(dev.T[None], device="cuda")
    D = negf.Device(Hd, Hu)
    Et = torch.as_tensor(E, device="cuda")
    st = torch.zeros(len(E), dtype=torch.int32, device="cuda")
    lead = negf.lead_selfenergy(D, Et, st, opt)
    kw = {}
    if sR is not None:
        kw = dict(scat_R=torch.as_tensor(sR, device="cuda"), scat_L=torch.as_tensor(sL, device="cuda"))
    Vbar, status = negf.rgf_adjoint(D, Et, st, lead["sigma_R"], lead["sigma_L"], opt,
                                    density_bar=torch.as_tensor(c, device="cuda"),
                                    current_bar=torch.as_tensor(d, device="cuda"),
                                    V=torch.as_tensor(V, device="cuda"), **kw)
    torch.cuda.synchronize()
    assert np.all(status.cpu().numpy() == 0)
    return Vbar.cpu().numpy(), (D, Et, st, lead, kw)


def _oracle_grad(dev, E, V, c, d, eta, sR=None, sL=None):
    N, b = dev.D.shape[0], dev.D.shape[1]
    g = np.zeros((N, b))
    for p, e in enumerate(E):
        leads = O.lead_self_energies(dev.D, dev.T, e, eta, 0.1, -0.1, O.KT_300K)
        g += O.gradient_dense(dev.D, dev.T, e, eta, V, leads, c[p], d[p],
                              None if sR is None else sR[p].reshape(N, b),
                              None if sL is None else sL[p].reshape(N, b))
    return g


@pytest.mark.parametrize("N,b,scatter", [(2, 3, False), (4, 6, False), (5, 8, True), (3, 40, True)])
def test_adjoint_matches_dense_gradient_fp64(N, b, scatter):
    dev, E, V, c, d, sR, sL = _setup(N, b, 900 + N * b, 4, scatter)
    g, _ = _gpu_grad(dev, E, V, c, d, negf.options(), sR, sL)
    ref = _oracle_grad(dev, E, V, c, d, 1e-6, sR, sL)
    # products of two Green's functions: roundoff grows with the square of the block condition
    assert np.abs(g - ref).max() <= 1e-7 * np.abs(ref).max()


def test_adjoint_mixed_precision():
    dev, E, V, c, d, sR, sL = _setup(4, 24, 77, 3, True)
    g, _ = _gpu_grad(dev, E, V, c, d, negf.options(precision=negf.PREC_MIXED), sR, sL)
    ref = _oracle_grad(dev, E, V, c, d, 1e-6, sR, sL)
    assert np.abs(g - ref).max() <= 1e-6 * np.abs(ref).max()


def test_adjoint_matches_gpu_finite_differences():
    N, b = 3, 5
    dev, E, V, c, d, sR, sL = _setup(N, b, 31, 2)
    opt = negf.options()
    g, (D, Et, st, lead, kw) = _gpu_grad(dev, E, V, c, d, opt)

    def loss(Vx):
        out = negf.rgf_solve(D, Et, st, lead["sigma_R"], lead["sigma_L"], opt,
                             V=torch.as_tensor(Vx, device="cuda"))
        n = out["density"].cpu().numpy()
        j = out["current"].cpu().numpy()
        return float((c * n).sum() + (d * j).sum())

    h = 1e-5
    for (i, q) in [(0, 0), (1, 2), (2, 4), (1, 0)]:
        Vp = V.copy()
        Vm = V.copy()
        Vp[i, q] += h
        Vm[i, q] -= h
        fd = (loss(Vp) - loss(Vm)) / (2 * h)
        assert abs(fd - g[i, q]) <= 1e-5 * max(np.abs(g).max(), 1e-12), (i, q, fd, g[i, q])


def test_adjoint_chunking_accumulates():
    dev, E, V, c, d, sR, sL = _setup(3, 7, 5, 5)
    g1, _ = _gpu_grad(dev, E, V, c, d, negf.options(chunk=2))
    g2, _ = _gpu_grad(dev, E, V, c, d, negf.options())
    assert np.abs(g1 - g2).max() <= 1e-12 * np.abs(g2).max()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("scatter", [False, True])
def test_adjoint_checkpointing_matches_stored_sweep(prec, scatter):
    """Sweep checkpointing (adjoint_segment = 1, 2, 3, 4 on N = 7 slabs: segments of one slab,
    even and uneven splits, a last segment of one slab) recomputes the same blocks, so V_bar
    agrees with the sweep that keeps every block; and with the dense oracle gradient."""
    N, b = 7, 12
    dev, E, V, c, d, sR, sL = _setup(N, b, 31, 3, scatter=scatter)
    g_all, _ = _gpu_grad(dev, E, V, c, d, negf.options(precision=prec), sR, sL)
    for seg in (1, 2, 3, 4):
        g_seg, _ = _gpu_grad(dev, E, V, c, d, negf.options(precision=prec, adjoint_segment=seg),
                             sR, sL)
        assert np.abs(g_seg - g_all).max() <= 1e-12 * np.abs(g_all).max(), seg
    g_ref = _oracle_grad(dev, E, V, c, d, 1e-6, sR, sL)
    # the bars of the dense-gradient tests above (products of two Green's functions)
    tol = 1e-7 if prec == 0 else 1e-5
    assert np.abs(g_all - g_ref).max() <= tol * np.abs(g_ref).max()


def test_autograd_function_uses_the_adjoint():
    dev, E, V, c, d, sR, sL = _setup(4, 6, 13, 3)
    opt = negf.options()
    g_ref, (D, Et, st, lead, kw) = _gpu_grad(dev, E, V, c, d, opt)
    Vt = torch.as_tensor(V, device="cuda").requires_grad_(True)
    dens, cur = negf.rgf(Vt, D, Et, st, lead["sigma_R"], lead["sigma_L"], opt)
    loss = (torch.as_tensor(c, device="cuda") * dens).sum() + \
        (torch.as_tensor(d, device="cuda") * cur).sum()
    loss.backward()
    assert np.abs(Vt.grad.cpu().numpy() - g_ref).max() <= 1e-12 * np.abs(g_ref).max()


def test_adjoint_finite_differences_on_16_atoms():
    """Reduced copy of the Newton-Poisson workload (N = 10 slabs x 343 orbitals, potential per
    atom of 10 orbitals): dL/dV_atom from the adjoint against central differences of the FP64
    GPU solve for 16 atoms, delta = 1e-4 eV."""
    from workloads import random_potential
    N, b = 10, 343
    dev = make_device(N, b, 4004)
    rng = np.random.default_rng(4)
    E = np.array([-0.45, 0.12])
    V = random_potential(N, b, 4504, 0.3)
    c = rng.normal(size=(len(E), N * b))
    d = rng.normal(size=(len(E), N - 1))
    opt = negf.options()
    g, (D, Et, st, lead, kw) = _gpu_grad(dev, E, V, c, d, opt)

    def loss(Vx):
        out = negf.rgf_solve(D, Et, st, lead["sigma_R"], lead["sigma_L"], opt,
                             V=torch.as_tensor(Vx, device="cuda"))
        return float((c * out["density"].cpu().numpy()).sum()
                     + (d * out["current"].cpu().numpy()).sum())

    h = 1e-4
    atoms = [(i, a) for i in range(0, N, 2) for a in (0, 11, 33)][:16]
    for (i, a) in atoms:
        sl = slice(10 * a, min(10 * a + 10, b))
        Vp = V.copy()
        Vm = V.copy()
        Vp[i, sl] += h
        Vm[i, sl] -= h
        fd = (loss(Vp) - loss(Vm)) / (2 * h)
        ga = g[i, sl].sum()
        assert abs(fd - ga) <= 1e-5 * max(abs(ga), 1e-3 * np.abs(g).max()), (i, a, fd, ga)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("scatter,chunk", [(False, 0), (True, 0), (True, 2)])
def test_adjoint_from_solve_checkpoints(prec, scatter, chunk):
    """negf_rgf_solve's checkpoints hand the sweep blocks to negf_rgf_adjoint: the same V_bar as
    the adjoint that recomputes them (same arithmetic, so to rounding), also when the solve and
    the adjoint split the points into different chunks."""
    N, b = 6, 20
    dev, E, V, c, d, sR, sL = _setup(N, b, 77, 5, scatter=scatter)
    opt = negf.options(precision=prec)
    g_ref, (D, Et, st, lead, kw) = _gpu_grad(dev, E, V, c, d, opt, sR, sL)
    ck = negf.checkpoint_buffer(D, len(E))
    Vt = torch.as_tensor(V, device="cuda")
    negf.rgf_solve(D, Et, st, lead["sigma_R"], lead["sigma_L"], negf.options(precision=prec),
                   V=Vt, checkpoints=ck, **kw)
    g, status = negf.rgf_adjoint(D, Et, st, lead["sigma_R"], lead["sigma_L"],
                                 negf.options(precision=prec, chunk=chunk),
                                 density_bar=torch.as_tensor(c, device="cuda"),
                                 current_bar=torch.as_tensor(d, device="cuda"), V=Vt,
                                 checkpoints=ck, **kw)
    torch.cuda.synchronize()
    assert np.all(status.cpu().numpy() == 0)
    assert np.abs(g.cpu().numpy() - g_ref).max() <= 1e-12 * np.abs(g_ref).max()


def test_autograd_keeps_the_sweeps():
    dev, E, V, c, d, sR, sL = _setup(4, 6, 13, 3)
    opt = negf.options()
    g_ref, (D, Et, st, lead, kw) = _gpu_grad(dev, E, V, c, d, opt)
    Vt = torch.as_tensor(V, device="cuda").requires_grad_(True)
    dens, cur = negf.rgf(Vt, D, Et, st, lead["sigma_R"], lead["sigma_L"], opt, keep_sweeps=True)
    loss = (torch.as_tensor(c, device="cuda") * dens).sum() + \
        (torch.as_tensor(d, device="cuda") * cur).sum()
    loss.backward()
    assert np.abs(Vt.grad.cpu().numpy() - g_ref).max() <= 1e-12 * np.abs(g_ref).max()
