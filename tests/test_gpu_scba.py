"""Self-consistent Born loop (Eqs. 4-6) on the GPU through the C ABI against the oracle loop:
20 Jacobi iterations of negf_rgf_solve (diag G^R, G^<) + negf_scba_step on a two-k device with
elastic acoustic and inelastic optical (E +- hw) scattering.

The device broadening is 1e-2 eV: with 1e-6 the undamped Jacobi iteration of this synthetic
device does not converge (quasi-bound states give |diag G| ~ 1/eta and the update overshoots),
so two correct implementations drift apart; with 1e-2 it contracts to |dSigma| ~ 3e-8."""
import numpy as np
import pytest

import oracle as O
from workloads import make_device, hamiltonian_k, k_grid, energy_grid_uniform

torch = pytest.importorskip("torch")
negf = pytest.importorskip("paper_1510_04686_gb300")

pytestmark = pytest.mark.gpu
ETA_DEV = 1e-2


@pytest.fixture(scope="module", autouse=True)
def _lib():
    negf._build.build()
    negf.library()


def _born(prec, iters=20, eta_dev=ETA_DEV, mix=1.0):
    N, b = 4, 6
    dev = make_device(N, b, 4321, with_k=True)
    ks, wk = k_grid(2)
    E, wE = energy_grid_uniform(-1.0, 0.05, 40)
    shift, hw, kT = 2, 0.10, O.KT_300K
    n0 = float(O.bose(hw, kT))
    Dac, Dop = 0.01, 0.02
    Hd = np.stack([hamiltonian_k(dev, float(k))[0] for k in ks])
    n_k, n_E, NB = len(ks), len(E), N * b
    # ---- oracle loop
    sR = np.zeros((n_E, NB), complex)
    sL = np.zeros_like(sR)
    for _ in range(iters):
        outs = [[O.solve_point(Hd[k], dev.T, E[j], eta_dev, None, eta_lead=1e-6, sR=sR[j].reshape(N, b),
                               sL=sL[j].reshape(N, b)) for j in range(n_E)] for k in range(n_k)]
        dGR = np.array([[o["diagGR"] for o in row] for row in outs])
        dGL = np.array([[o["diagGL"] for o in row] for row in outs])
        sR, sL, delta = O.scba_step(dGR, dGL, wk, Dac, Dop, shift, n0, sR, sL, mix=mix)
    dens_ref = np.array([[o["density"] for o in row] for row in outs])
    # ---- GPU loop
    D = negf.Device(torch.as_tensor(Hd, device="cuda"),
                    torch.as_tensor(np.stack([dev.T] * n_k), device="cuda"))
    Et = torch.as_tensor(np.tile(E, n_k), device="cuda")
    st = torch.as_tensor(np.repeat(np.arange(n_k), n_E).astype(np.int32), device="cuda")
    ei = torch.as_tensor(np.tile(np.arange(n_E), n_k).astype(np.int32), device="cuda")
    opt = negf.options(precision=prec, eta_device=eta_dev)
    lead = negf.lead_selfenergy(D, Et, st, opt)
    gR = torch.zeros((n_E, NB), dtype=torch.complex128, device="cuda")
    gL = torch.zeros_like(gR)
    wkt = torch.as_tensor(wk, device="cuda")
    for _ in range(iters):
        out = negf.rgf_solve(D, Et, st, lead["sigma_R"], lead["sigma_L"], opt, scat_R=gR,
                             scat_L=gL, e_idx=ei, diag=True, outputs=("density",))
        d_gpu = negf.scba_step(out["diagGR"].reshape(n_k, n_E, NB),
                               out["diagGL"].reshape(n_k, n_E, NB), wkt, gR, gL, Dac, Dop, shift,
                               n0, mix)
    torch.cuda.synchronize()
    return (sR, sL, delta, dens_ref.reshape(n_k * n_E, NB), gR.cpu().numpy(), gL.cpu().numpy(),
            float(d_gpu.cpu()), out["density"].cpu().numpy())


# The Born map of this device amplifies a 1e-14 perturbation of the first iterate to ~3e-8
# after 20 iterations (measured with the oracle alone), so two correct FP64 loops agree to
# ~1e-13 after 8 iterations but only to ~1e-7 after 20; the bounds below follow that growth.
@pytest.mark.parametrize("prec,iters,tol", [(0, 8, 1e-9), (1, 8, 1e-6), (0, 20, 1e-5),
                                             (1, 20, 1e-5)])
def test_born_loop_matches_oracle(prec, iters, tol):
    sR, sL, delta, dens_ref, gR, gL, dgpu, dens = _born(prec, iters)
    assert np.abs(gR - sR).max() <= tol * np.abs(sR).max()
    assert np.abs(gL - sL).max() <= tol * np.abs(sL).max()
    assert np.abs(dens - dens_ref).max() <= tol * np.abs(dens_ref).max()
    if iters == 20:
        assert delta < 1e-6  # the loop converged
    assert abs(dgpu - delta) <= 1e-3 * max(delta, 1e-12) + tol * np.abs(sR).max()


# At the benchmark's device broadening (1e-6 eV) the damped iteration (mixing 0.5) contracts on
# this device (|dSigma| 9e-2, 6.5e-2, 2.1e-2, 8.3e-3, 6.2e-3 over five updates) and a 1e-14
# perturbation of the lead self-energies moves the fifth iterate by ~1e-13 (oracle alone), so two
# correct loops agree to rounding there; the bars are those of the per-point sweep parity.
@pytest.mark.parametrize("prec,tol", [(0, 1e-9), (1, 1e-6)])
def test_damped_born_loop_at_the_benchmark_broadening(prec, tol):
    sR, sL, delta, dens_ref, gR, gL, dgpu, dens = _born(prec, 5, eta_dev=1e-6, mix=0.5)
    assert np.abs(gR - sR).max() <= tol * np.abs(sR).max()
    assert np.abs(gL - sL).max() <= tol * np.abs(sL).max()
    assert np.abs(dens - dens_ref).max() <= tol * np.abs(dens_ref).max()
    assert abs(dgpu - delta) <= 1e-3 * delta + tol * np.abs(sR).max()
