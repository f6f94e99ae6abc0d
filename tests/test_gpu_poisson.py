"""NEGF-Poisson self-consistency (Eq. 9) on the GPU against the oracle.

The Poisson residual and the orbital/atom maps are compared with the oracle's plain loops; the
Newton loop (densities by the RGF sweeps, Jacobian rows by the adjoint sweep, Newton step by the
library's FP64 block inverse) is run on a reduced copy of the adjoint workload's device and must
converge to the oracle loop's potential (the oracle differentiates by the dense definition)."""
import numpy as np
import pytest

import oracle as O
from workloads import config_workload, make_device

torch = pytest.importorskip("torch")
negf = pytest.importorskip("paper_1510_04686_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    negf._build.build()
    negf.library()


def _t(x):
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


@pytest.mark.parametrize("N,A", [(7, 6), (5, 1), (4, 2)])
def test_poisson_apply_matches_oracle(N, A):
    rng = np.random.default_rng(N * 10 + A)
    U, n, nD = rng.normal(size=(N, A)), rng.random((N, A)) * 5, rng.random((N, A)) * 5
    args = (1.3, 0.4, 0.2, -0.15, 0.07)
    F = negf.poisson_apply(_t(U), *args[:4], kappa=args[4], n=_t(n), n_D=_t(nD)).cpu().numpy()
    ref = O.poisson_residual(U, n, nD, *args)
    assert np.abs(F - ref).max() < 1e-13
    K = negf.poisson_apply(_t(U), 1.3, 0.4).cpu().numpy()
    assert np.abs(K - O.poisson_residual(U, None, None, 1.3, 0.4, 0.0, 0.0, 0.0)).max() < 1e-13


@pytest.mark.parametrize("b", [40, 35])
def test_orbital_atom_maps_match_oracle(b):
    N = 3
    rng = np.random.default_rng(b)
    orb = rng.normal(size=(2, N * b))
    at = negf.orbitals_to_atoms(_t(orb), N, b).cpu().numpy()
    for g in range(2):
        assert np.abs(at[g] - O.atom_sums(orb[g], N, b)).max() < 1e-13
    U = rng.normal(size=(N, -(-b // 10)))
    assert np.array_equal(negf.atoms_to_orbitals(_t(U), b).cpu().numpy(),
                          O.atom_to_orbitals(U, b))


@pytest.mark.parametrize("prec", [0, 1])
def test_newton_poisson_matches_oracle_loop(prec):
    """Reduced adjoint workload (N = 4 slabs, b = 40: 16 atoms, 16 energies over [-3, 3] eV),
    eta = 0.05 eV (a broadening that the 0.4 eV energy grid resolves, so that n(U) is smooth
    enough for Newton; at eta = 1e-3 the oracle loop itself does not converge on this grid),
    contacts grounded, donors 0.2 electrons per atom above the mean electrons of the flat
    potential: the GPU Newton loop reaches max |F| < 1e-10 (FP64; 1e-8 mixed) and its potential
    equals the oracle loop's within 1e-9 (FP64) or 1e-6 (mixed) eV."""
    w = config_workload(4, N=4, b=40, n_E=16)
    dev, E, wE = w["device"], w["E"], w["wE"]
    N, b, A, eta = 4, 40, 4, 0.05
    cx, cy, kappa = 1.0, 0.5, 0.05
    leads = [O.lead_self_energies(dev.D, dev.T, float(e), eta, 0.1, -0.1, O.KT_300K) for e in E]
    n0 = O.electrons_per_atom(dev.D, dev.T, E, wE, eta, np.zeros((N, A)), leads)
    nD = np.full((N, A), n0.mean()) + 0.2
    U_ref, hist_ref = O.poisson_newton(dev.D, dev.T, E, wE, eta, nD, cx, cy, 0.0, 0.0, kappa,
                                       tol=1e-11)
    assert hist_ref[-1] < 1e-11
    d = negf.Device(_t(dev.D[None]), _t(dev.T[None]))
    opt = negf.options(precision=prec, eta_lead=eta, eta_device=eta)
    U, hist = negf.poisson_newton(d, _t(E), _t(wE), torch.zeros(len(E), dtype=torch.int32,
                                                               device="cuda"),
                                  opt, _t(nD), kappa, cx, cy,
                                  tol=1e-10 if prec == 0 else 1e-8)
    U = U.cpu().numpy()
    print(f"precision {prec}: residuals {['%.1e' % h for h in hist]}, "
          f"|U - U_oracle| {np.abs(U - U_ref).max():.2e}, |U| {np.abs(U_ref).max():.2e}")
    assert hist[-1] < (1e-10 if prec == 0 else 1e-8) and len(hist) <= 10
    assert np.abs(U - U_ref).max() < (1e-9 if prec == 0 else 1e-6)
