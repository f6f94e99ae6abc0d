"""Pins of the CPU oracle against facts fixed by the paper and by the mathematics.

Each test checks the oracle against something other than itself: dense inversion of Eq. (1)-(2),
closed forms of the 1D tight-binding chain, channel counting, current conservation, the
fluctuation-dissipation relation, the algebraic identity behind Eq. (6), and finite differences.
"""
import numpy as np
import pytest

import oracle as O
from workloads import make_device, chain_device, channel_device

KT = O.KT_300K


def _scatter(N, b, seed, gamma=0.05, f=0.7):
    """Physical orbital-diagonal self-energies: Sigma^R = r - i g, Sigma^< = i f 2 g."""
    rng = np.random.default_rng(seed)
    g = gamma * rng.random((N, b))
    r = 0.02 * rng.normal(size=(N, b))
    sR = r - 1j * g
    sL = 1j * f * 2 * g
    return sR, sL


def _blocks(M, N, b):
    diag = [M[i * b:(i + 1) * b, i * b:(i + 1) * b] for i in range(N)]
    lower = [M[(i + 1) * b:(i + 2) * b, i * b:(i + 1) * b] for i in range(N - 1)]
    return diag, lower


@pytest.mark.parametrize("N,b", [(1, 3), (2, 1), (3, 4), (6, 5)])
@pytest.mark.parametrize("scatter", [False, True])
def test_rgf_equals_dense_inverse(N, b, scatter):
    dev = make_device(N, b, 11 + N * b)
    V = np.random.default_rng(5).uniform(-0.3, 0.3, (N, b))
    E, eta = 0.37, 1e-6
    leads = O.lead_self_energies(dev.D, dev.T, E, eta, 0.1, -0.1, KT)
    sR, sL = _scatter(N, b, 3) if scatter else (None, None)
    r = O.rgf(dev.D, dev.T, E, eta, V, leads, sR, sL)
    G, GL = O.dense_green(dev.D, dev.T, E, eta, V, leads, sR, sL)
    Gd, _ = _blocks(G, N, b)
    GLd, GLl = _blocks(GL, N, b)
    scale = max(np.abs(G).max(), 1.0)
    scale_l = max(np.abs(GL).max(), 1e-300)
    for i in range(N):
        assert np.abs(r["G"][i] - Gd[i]).max() < 1e-11 * scale
        assert np.abs(r["GL"][i] - GLd[i]).max() < 1e-11 * scale_l
    for i in range(N - 1):
        assert np.abs(r["GLoff"][i] - GLl[i]).max() < 1e-11 * scale_l


def _chain_surface_closed_form(z, eps, t):
    disc = np.sqrt((z - eps) ** 2 - 4 * t * t + 0j)
    roots = [((z - eps) + disc) / (2 * t * t), ((z - eps) - disc) / (2 * t * t)]
    # the retarded surface Green's function is the root with |t g| < 1 (decaying into the lead)
    return min(roots, key=lambda g: abs(t * g))


@pytest.mark.parametrize("E", [-2.7, -1.3, -0.41, 0.2, 0.93, 1.999, 2.4])
def test_sancho_rubio_chain_closed_form(E):
    eps, t, eta = 0.0, 1.0, 1e-9
    z = E + 1j * eta
    gs, it, conv = O.sancho_rubio(np.array([[eps]]), np.array([[t]]), z)
    assert conv and it < 100
    exact = _chain_surface_closed_form(z, eps, t)
    assert abs(gs[0, 0] - exact) < 2e-6 * max(1.0, abs(exact))
    assert gs[0, 0].imag <= 1e-12


def test_sancho_rubio_fixed_point_and_causality():
    rng = np.random.default_rng(7)
    b = 6
    h = rng.normal(size=(b, b)) + 1j * rng.normal(size=(b, b))
    h = 0.3 * (h + h.conj().T)
    a = (rng.normal(size=(b, b)) + 1j * rng.normal(size=(b, b))) / np.sqrt(2 * b)
    for E in [-1.1, 0.05, 0.8]:
        z = E + 1j * 1e-6
        gs, it, conv = O.sancho_rubio(h, a, z)
        assert conv
        resid = gs - np.linalg.inv(z * np.eye(b) - h - a @ gs @ a.conj().T)
        assert np.abs(resid).max() < 1e-8 * max(1.0, np.abs(gs).max())
        spec = np.linalg.eigvalsh(1j * (gs - gs.conj().T))
        assert spec.min() > -1e-9 * max(1.0, np.abs(spec).max())


def test_sancho_rubio_matches_long_finite_lead():
    """With eta = 0.05 a lead of 3000 cells is indistinguishable from a semi-infinite one."""
    rng = np.random.default_rng(8)
    b = 3
    h = rng.normal(size=(b, b)) + 1j * rng.normal(size=(b, b))
    h = 0.25 * (h + h.conj().T)
    a = (rng.normal(size=(b, b)) + 1j * rng.normal(size=(b, b))) / np.sqrt(2 * b)
    z = 0.3 + 0.05j
    g = np.linalg.inv(z * np.eye(b) - h)
    for _ in range(3000):
        g = np.linalg.inv(z * np.eye(b) - h - a @ g @ a.conj().T)
    gs, _, conv = O.sancho_rubio(h, a, z)
    assert conv
    assert np.abs(gs - g).max() < 1e-10 * np.abs(g).max()


@pytest.mark.parametrize("E", [-2.5, -1.7, -0.3, 0.6, 1.95, 2.2, 3.1])
def test_transmission_chain_is_step(E):
    ch = chain_device(7, 0.0, 1.0)
    o = O.solve_point(ch.D, ch.T, E, 0.0, None, eta_lead=1e-9)
    expected = 1.0 if abs(E) < 2.0 else 0.0
    assert abs(o["transmission"] - expected) < 1e-6


def test_transmission_channel_counting():
    dev = channel_device(4, 5, 21)
    d, t = dev.meta["d"], dev.meta["t"]
    for E in np.linspace(-3.2, 3.2, 41):
        dist = np.abs(np.abs(E - d) - 2 * t)
        if dist.min() < 1e-3:
            continue
        count = int(np.sum(np.abs(E - d) < 2 * t))
        o = O.solve_point(dev.D, dev.T, E, 0.0, None, eta_lead=1e-9)
        assert abs(o["transmission"] - count) < 1e-5, (E, o["transmission"], count)


def test_caroli_equals_gnn_formula():
    dev = make_device(5, 4, 31)
    for E in [-1.0, 0.1, 1.2]:
        o = O.solve_point(dev.D, dev.T, E, 0.0, None, eta_lead=1e-7)
        G, _ = O.dense_green(dev.D, dev.T, E, 0.0, None, o["leads"])
        Tc = O.transmission_caroli_dense(G, o["leads"]["gamL"], o["leads"]["gamR"], 5, 4)
        assert abs(Tc - o["transmission"]) < 1e-9 * max(1.0, Tc)


def test_current_conservation_and_landauer():
    dev = make_device(6, 4, 41)
    V = np.random.default_rng(2).uniform(-0.2, 0.2, (6, 4))
    for E in [-0.8, -0.05, 0.07, 0.9]:
        o = O.solve_point(dev.D, dev.T, E, 0.0, V, eta_lead=1e-7, mu_L=0.1, mu_R=-0.1)
        j = o["current"]
        df = O.fermi(E, 0.1, KT) - O.fermi(E, -0.1, KT)
        land = df * o["transmission"]
        assert np.abs(j - land).max() < 1e-9 * max(abs(land), 1e-12) + 1e-13
        assert land >= -1e-15  # positive for left-to-right flow (mu_L > mu_R)
        o0 = O.solve_point(dev.D, dev.T, E, 0.0, V, eta_lead=1e-7, mu_L=0.05, mu_R=0.05)
        assert np.abs(o0["current"]).max() < 1e-12


def test_fluctuation_dissipation_equilibrium():
    N, b = 5, 4
    dev = make_device(N, b, 51)
    mu = 0.02
    for E in [-0.5, 0.03, 0.4]:
        f = float(O.fermi(E, mu, KT))
        # equilibrium elastic scattering: Sigma^< = -f (Sigma^R - Sigma^A)
        rng = np.random.default_rng(3)
        gam = 0.03 * rng.random((N, b))
        sR = 0.01 * rng.normal(size=(N, b)) - 1j * gam
        sL = 1j * f * 2 * gam
        # eta only in the leads: a device eta would broaden A without feeding Sigma^<
        o = O.solve_point(dev.D, dev.T, E, 0.0, None, eta_lead=1e-6, mu_L=mu, mu_R=mu, sR=sR,
                          sL=sL)
        for Gi, GLi in zip(o["blocks"]["G"], o["blocks"]["GL"]):
            ref = -f * (Gi - Gi.conj().T)
            assert np.abs(GLi - ref).max() < 1e-9 * max(np.abs(ref).max(), 1e-12)


def test_spectral_function_hermitian_psd_and_lesser_antihermitian():
    N, b = 6, 5
    dev = make_device(N, b, 61)
    sR, sL = _scatter(N, b, 9)
    for E in [-1.3, 0.0123, 0.77]:
        o = O.solve_point(dev.D, dev.T, E, 1e-6, None, sR=sR, sL=sL)
        for Gi, GLi in zip(o["blocks"]["G"], o["blocks"]["GL"]):
            A = 1j * (Gi - Gi.conj().T)
            assert np.abs(A - A.conj().T).max() == 0.0 or np.abs(A - A.conj().T).max() < 1e-14
            w = np.linalg.eigvalsh(A)
            assert w.min() > -1e-12 * np.abs(w).max()
            assert np.abs(GLi + GLi.conj().T).max() < 1e-12 * max(np.abs(GLi).max(), 1e-300)
        assert o["density"].min() > -1e-14


def test_bose_occupation_at_300K():
    # n0 = 1/(exp(hw/kT) - 1) for hw = 60 meV, kT = 25.852 meV is 0.10887 (closed form)
    assert abs(O.bose(0.060, KT) - 1.0 / (np.exp(0.060 / KT) - 1.0)) < 1e-15
    assert abs(O.bose(0.060, KT) - 0.108869) < 1e-5


def test_scba_reduces_to_ballistic_and_truncates():
    rng = np.random.default_rng(4)
    n_k, n_E, n_orb = 3, 30, 7
    dGR = rng.normal(size=(n_k, n_E, n_orb)) + 1j * rng.normal(size=(n_k, n_E, n_orb))
    dGL = 1j * rng.random((n_k, n_E, n_orb))
    wk = np.full(n_k, 1.0 / n_k)
    sR, sL = O.scba_selfenergy(dGR, dGL, wk, 0.0, 0.0, 12, 0.1)
    assert np.all(sR == 0) and np.all(sL == 0)
    # a single nonzero energy j0 feeds the optical terms only at j0 +- shift
    dGR[:] = 0
    dGL[:] = 0
    j0, sh = 15, 4
    dGR[:, j0, :] = 1.0 + 2.0j
    dGL[:, j0, :] = 3.0j
    sR, sL = O.scba_selfenergy(dGR, dGL, wk, 0.0, 0.5, sh, 0.25)
    nz_R = sorted(set(np.nonzero(np.abs(sR).max(axis=1))[0].tolist()))
    nz_L = sorted(set(np.nonzero(np.abs(sL).max(axis=1))[0].tolist()))
    assert nz_R == [j0 - sh, j0 + sh] and nz_L == [j0 - sh, j0 + sh]
    # emission (E -> E - hw) carries 1 + n0, absorption carries n0 (Eq. 5)
    assert np.allclose(sL[j0 - sh], 0.5 * 1.25 * 3.0j)
    assert np.allclose(sL[j0 + sh], 0.5 * 0.25 * 3.0j)
    # energies shifted off the grid contribute nothing
    dGL[:] = 0
    dGL[:, 1, :] = 1j
    sR, sL = O.scba_selfenergy(dGR * 0, dGL, wk, 0.0, 1.0, 5, 0.1)
    assert np.abs(sL[0]).max() == 0.0 and np.abs(sL[6]).max() > 0


def test_scba_retarded_antihermitian_part_is_half_greater_minus_lesser():
    """Eq. (6) (comma read as '+') has anti-Hermitian part (Sigma^> - Sigma^<) / 2 exactly.

    Built independently: G^> = G^R - G^A + G^<, and Sigma^> of the optical phonon takes
    (1+n0) G^>(E-hw) + n0 G^>(E+hw); the acoustic one D_ac G^>(E).
    """
    rng = np.random.default_rng(12)
    n_k, n_E, n_orb, sh = 2, 40, 5, 6
    n0, Dac, Dop = 0.1089, 0.01, 0.02
    gam = rng.random((n_k, n_E, n_orb))
    f = rng.random((n_k, n_E, n_orb))
    dGR = 0.3 * rng.normal(size=gam.shape) - 1j * gam       # diag G^R
    dGL = 1j * f * 2 * gam                                    # diag G^< = i f A
    dGG = dGR - dGR.conj() + dGL                               # diag G^>
    wk = np.array([0.3, 0.7])
    sR, sL = O.scba_selfenergy(dGR, dGL, wk, Dac, Dop, sh, n0)
    sumG = np.einsum("k,kej->ej", wk, dGG)
    sumL = np.einsum("k,kej->ej", wk, dGL)

    def at(a, j):
        return a[j] if 0 <= j < n_E else 0 * a[0]

    for j in range(n_E):
        sG = Dac * sumG[j] + Dop * ((1 + n0) * at(sumG, j - sh) + n0 * at(sumG, j + sh))
        sLj = Dac * sumL[j] + Dop * ((1 + n0) * at(sumL, j + sh) + n0 * at(sumL, j - sh))
        anti = 0.5 * (sR[j] - sR[j].conj())
        assert np.allclose(anti, 0.5 * (sG - sLj), atol=1e-14)
        assert np.allclose(sL[j], sLj, atol=1e-14)


def test_gradient_dense_matches_finite_differences():
    N, b = 3, 3
    dev = make_device(N, b, 71)
    rng = np.random.default_rng(6)
    V = rng.uniform(-0.2, 0.2, (N, b))
    c = rng.normal(size=(N * b))
    d = rng.normal(size=(N - 1))
    E, eta = 0.21, 1e-3
    leads = O.lead_self_energies(dev.D, dev.T, E, eta, 0.1, -0.1, KT)

    def loss(Vx):
        r = O.rgf(dev.D, dev.T, E, eta, Vx, leads)
        return float(c @ O.density_from_blocks(r["GL"]) + d @ O.current_from_blocks(dev.T, r["GLoff"]))

    g = O.gradient_dense(dev.D, dev.T, E, eta, V, leads, c, d)
    h = 1e-5
    fd = np.zeros_like(V)
    for i in range(N):
        for j in range(b):
            Vp = V.copy()
            Vm = V.copy()
            Vp[i, j] += h
            Vm[i, j] -= h
            fd[i, j] = (loss(Vp) - loss(Vm)) / (2 * h)
    assert np.abs(g - fd).max() < 1e-6 * np.abs(fd).max()


def test_acoustic_scba_conserves_current_per_energy():
    """Elastic (acoustic) scattering conserves the bond current at every energy at convergence.

    Clean channels with every channel open keep all states coupled to the leads, so the Born
    iteration converges with no device eta (a device eta would leak current).
    """
    N, b = 5, 3
    dev = channel_device(N, b, 21)
    E = np.linspace(-0.2, 0.2, 5)
    assert all(np.all(np.abs(e - dev.meta["d"]) < 2 * dev.meta["t"]) for e in E)
    sR = np.zeros((len(E), N * b), dtype=complex)
    sL = np.zeros_like(sR)
    for _ in range(200):
        outs = [O.solve_point(dev.D, dev.T, e, 0.0, None, eta_lead=1e-7, sR=sR[i].reshape(N, b),
                              sL=sL[i].reshape(N, b)) for i, e in enumerate(E)]
        dGR = np.array([o["diagGR"] for o in outs])[None]
        dGL = np.array([o["diagGL"] for o in outs])[None]
        sR, sL, delta = O.scba_step(dGR, dGL, np.ones(1), 0.05, 0.0, 3, 0.1, sR, sL)
        if delta < 1e-14:
            break
    assert delta < 1e-12
    for o in outs:
        j = o["current"]
        assert np.abs(j - j.mean()).max() < 1e-9 * max(np.abs(j).max(), 1e-12)
    # scattering changes the current relative to the ballistic Landauer value
    o_b = O.solve_point(dev.D, dev.T, E[2], 0.0, None, eta_lead=1e-7)
    assert abs(outs[2]["current"][0] - o_b["current"][0]) > 1e-6 * abs(o_b["current"][0])


def _born_fdt_violation(dev, E_max, shift, n_iter=2, dE=0.02, D_ac=0.002, D_op=0.004):
    """Max over energies of |G^<_jj - i f A_jj| / max_j |A_jj| after n_iter Born updates at
    equilibrium (mu_L = mu_R = 0, no device eta)."""
    E = np.arange(-E_max, E_max + dE / 2, dE)
    N, b = dev.N, dev.b
    n0 = O.bose(abs(shift) * dE, KT)
    sR = np.zeros((len(E), N * b), dtype=complex)
    sL = np.zeros_like(sR)
    for _ in range(n_iter + 1):
        outs = [O.solve_point(dev.D, dev.T, e, 0.0, None, eta_lead=1e-7, mu_L=0.0, mu_R=0.0,
                              kT=KT, sR=sR[i].reshape(N, b), sL=sL[i].reshape(N, b))
                for i, e in enumerate(E)]
        dGR = np.array([o["diagGR"] for o in outs])[None]
        dGL = np.array([o["diagGL"] for o in outs])[None]
        sR, sL, _ = O.scba_step(dGR, dGL, np.ones(1), D_ac, D_op, shift, n0, sR, sL)
    f = 1.0 / (np.exp(E / KT) + 1.0)
    worst = 0.0
    for i, o in enumerate(outs):
        A = 1j * (o["diagGR"] - o["diagGR"].conj())
        worst = max(worst, np.abs(o["diagGL"] - 1j * f[i] * A).max() / np.abs(A).max())
    return worst


def test_scba_keeps_equilibrium_detailed_balance():
    """At equilibrium every Born update of Eqs. (4)-(6) keeps G^< = -f (G^R - G^A) = i f A.

    If G^< = i f A at all energies, the optical terms pair (1 + n0) G^<(E + hw) in Sigma^< with
    n0 G^>(E + hw) in Sigma^> (and n0 G^<(E - hw) with (1 + n0) G^>(E - hw)).  Fermi and Bose
    factors at one temperature satisfy (1 + n0) f(E + hw) (1 - f(E)) = n0 (1 - f(E + hw)) f(E),
    so every pair obeys the KMS relation Sigma^< (1 - f) = -f Sigma^> on its own (grid
    truncation drops whole pairs), and the next G^< = G^R Sigma^< G^A is i f A again: the check
    is exact at every energy.  Exchanging emission and absorption (the sign of the energy shift,
    a mistake planted here in the oracle's input) breaks it.
    """
    for dev, E_max in ((chain_device(6, 0.0, 0.1), 0.6),
                       (channel_device(4, 3, 21, d_lo=-0.1, d_hi=0.1), 0.8)):
        assert _born_fdt_violation(dev, E_max, 3) < 1e-12
        assert _born_fdt_violation(dev, E_max, -3) > 1e-4


def _optical_born_currents(dev, n0_lesser_factor=1.0, shift=3, dE=0.02, E_max=0.8, D_op=0.004):
    """Born loop with optical phonons only (Eqs. 5-6) at the default bias, to |dSigma| < 1e-12;
    returns the bond currents j_i(E).  n0_lesser_factor != 1 plants a mistake in the oracle's
    update: Sigma^< then uses another phonon occupation than Sigma^R."""
    E = np.arange(-E_max, E_max + dE / 2, dE)
    N, b = dev.N, dev.b
    n0 = O.bose(shift * dE, KT)
    sR = np.zeros((len(E), N * b), dtype=complex)
    sL = np.zeros_like(sR)

    def solve():
        return [O.solve_point(dev.D, dev.T, e, 0.0, None, eta_lead=1e-7, sR=sR[i].reshape(N, b),
                              sL=sL[i].reshape(N, b)) for i, e in enumerate(E)]

    for _ in range(60):
        outs = solve()
        dGR = np.array([o["diagGR"] for o in outs])[None]
        dGL = np.array([o["diagGL"] for o in outs])[None]
        nR, nL = O.scba_selfenergy(dGR, dGL, np.ones(1), 0.0, D_op, shift, n0)
        if n0_lesser_factor != 1.0:
            _, nL = O.scba_selfenergy(dGR, dGL, np.ones(1), 0.0, D_op, shift, n0_lesser_factor * n0)
        delta = max(np.abs(nR - sR).max(), np.abs(nL - sL).max())
        sR, sL = nR, nL
        if delta < 1e-12:
            break
    assert delta < 1e-12
    return np.array([o["current"] for o in solve()]), dE


def test_optical_scba_conserves_energy_integrated_current():
    """Inelastic scattering moves electrons between energies, so j_i(E) differs from bond to bond,
    but at convergence of Eqs. (5)-(6) no particle is lost: the energy integral of j_i is the
    same on every bond.  Each in-scattering term of Sigma^<(E) from E +- hw meets the matching
    out-scattering term of Sigma^>(E +- hw) (energies shifted off the grid drop both), so the
    balance is exact.  A Sigma^< whose phonon occupation differs from that of Sigma^R (planted)
    breaks it."""
    dev = channel_device(4, 3, 21, d_lo=-0.1, d_hi=0.1)
    J, dE = _optical_born_currents(dev)
    J_int = J.sum(axis=0) * dE
    assert np.abs(J_int - J_int.mean()).max() < 1e-10 * np.abs(J_int).max()
    assert np.abs(J - J.mean(axis=1, keepdims=True)).max() > 1e-4 * np.abs(J).max()
    J_bad, _ = _optical_born_currents(dev, n0_lesser_factor=2.0)
    J_bad_int = J_bad.sum(axis=0) * dE
    assert np.abs(J_bad_int - J_bad_int.mean()).max() > 1e-3 * np.abs(J_bad_int).max()


def test_density_sum_rule_fixes_eq7_normalisation():
    """Eq. (7)'s n_j(E) = Im G^<_jj(E) / 2 pi integrates to the occupation of orbital j.

    Every state of a chain lies in |E| < 2t, and the local density of states A_jj(E) of the
    open chain integrates to 2 pi (completeness).  With the band filled (mu far above it),
    integral n_j dE = 1 for every site; at mu = 0, particle-hole symmetry (A(-E) = A(E),
    f(-E) = 1 - f(E)) gives exactly 1/2.  The substitution E = 2t sin(theta) removes the band-edge
    singularities of A, so Gauss-Legendre nodes in theta integrate to ~1e-11.
    """
    t = 1.0
    dev = chain_device(5, 0.0, t)
    x, w = np.polynomial.legendre.leggauss(16)
    theta, w_theta = 0.5 * np.pi * x, 0.5 * np.pi * w
    E, wE = 2 * t * np.sin(theta), w_theta * 2 * t * np.cos(theta)
    for mu, expect in ((10.0, 1.0), (0.0, 0.5)):
        n = sum(we * O.solve_point(dev.D, dev.T, e, 0.0, None, eta_lead=1e-12, mu_L=mu, mu_R=mu,
                                   kT=KT)["density"] for e, we in zip(E, wE))
        assert np.abs(n - expect).max() < 1e-9


def test_integrate_is_the_trapezoid_rule_on_polynomials():
    """Eq. 7's energy quadrature with trapezoid weights integrates 1 and E exactly and E^2 with
    the closed-form trapezoid error h^2 (b - a) / 12 * 2 = h^2 on [-3, 3]; summation is in point
    order with the weights applied once."""
    from workloads import energy_grid_linspace
    for n in (5, 64, 513):
        E, w = energy_grid_linspace(-3.0, 3.0, n)
        h = 6.0 / (n - 1)
        vals = np.stack([np.ones(n), E, E ** 2, 2.0 * E ** 2 - 3.0], axis=1)
        out = O.integrate(vals, w)
        assert abs(out[0] - 6.0) < 1e-13
        assert abs(out[1]) < 1e-13
        assert abs(out[2] - (18.0 + h ** 2)) < 1e-12
        assert abs(out[3] - (2.0 * (18.0 + h ** 2) - 18.0)) < 1e-12
    # groups of points are integrated separately when the caller splits them
    E, w = energy_grid_linspace(-1.0, 1.0, 9)
    assert abs(O.integrate(np.ones((9, 1)), w)[0] - 2.0) < 1e-14


def test_scba_mixing_is_linear_with_a_fixed_point():
    """The Born update with linear mixing: Sigma <- (1 - m) Sigma_old + m Sigma_Born.  A Sigma_old
    that is already the Born self-energy of the given G is a fixed point for every m (delta 0);
    otherwise the step and the reported max |Delta Sigma| scale exactly with m."""
    rng = np.random.default_rng(12)
    n_k, n_E, n_orb = 2, 40, 5
    dGR = rng.normal(size=(n_k, n_E, n_orb)) + 1j * rng.normal(size=(n_k, n_E, n_orb))
    dGL = 1j * rng.random((n_k, n_E, n_orb))
    wk = np.array([0.25, 0.75])
    args = (dGR, dGL, wk, 0.01, 0.02, 12, O.bose(0.06, O.KT_300K))
    bornR, bornL = O.scba_selfenergy(*args)
    for m in (0.3, 1.0):
        nR, nL, d = O.scba_step(*args, bornR, bornL, mix=m)
        assert np.allclose(nR, bornR, atol=1e-15) and np.allclose(nL, bornL, atol=1e-15)
        assert d < 1e-15
    oldR = bornR + 0.1 * (rng.normal(size=bornR.shape) + 1j * rng.normal(size=bornR.shape))
    oldL = bornL + 0.1j * rng.random(bornL.shape)
    r1R, r1L, d1 = O.scba_step(*args, oldR, oldL, mix=1.0)
    r3R, r3L, d3 = O.scba_step(*args, oldR, oldL, mix=0.3)
    assert np.allclose(r1R, bornR) and np.allclose(r1L, bornL)
    assert np.allclose(r3R - oldR, 0.3 * (bornR - oldR), atol=1e-14)
    assert np.allclose(r3L - oldL, 0.3 * (bornL - oldL), atol=1e-14)
    assert abs(d3 - 0.3 * d1) < 1e-14


# ---- Eq. 9: NEGF-Poisson self-consistency -----------------------------------------------------

def test_poisson_operator_fourier_modes_and_linear_drop():
    """The finite-difference operator of Eq. 9 on the atom grid: a mode sin(pi m (i+1)/(N+1))
    cos(2 pi q a / A) with grounded contacts is an eigenvector with eigenvalue
    cx (2 - 2 cos(pi m / (N+1))) + cy (2 - 2 cos(2 pi q / A)) (both directions and the periodic
    wrap), and the contact-to-contact linear drop U_i = UL + (UR - UL)(i+1)/(N+1) has zero
    residual."""
    N, A, cx, cy = 7, 6, 1.3, 0.4
    i = np.arange(N)[:, None]
    a = np.arange(A)[None, :]
    for m, q in ((1, 0), (2, 1), (5, 3)):
        U = np.sin(np.pi * m * (i + 1) / (N + 1)) * np.cos(2 * np.pi * q * a / A)
        lam = cx * (2 - 2 * np.cos(np.pi * m / (N + 1))) + cy * (2 - 2 * np.cos(2 * np.pi * q / A))
        F = O.poisson_residual(U, None, None, cx, cy, 0.0, 0.0, 0.0)
        assert np.allclose(F, lam * U, atol=1e-13)
    UL, UR = 0.25, -0.35
    lin = np.repeat((UL + (UR - UL) * (np.arange(N) + 1) / (N + 1))[:, None], A, axis=1)
    assert np.abs(O.poisson_residual(lin, None, None, cx, cy, UL, UR, 0.0)).max() < 1e-14
    # the matrix form agrees with the residual's linear part
    K = O.poisson_matrix(N, A, cx, cy)
    U = np.random.default_rng(2).normal(size=(N, A))
    assert np.allclose(K @ U.ravel(), O.poisson_residual(U, None, None, cx, cy, 0, 0, 0).ravel())
    assert np.allclose(K, K.T)


def test_poisson_manufactured_solution_fixes_the_charge_term():
    """F(U*) = 0 for any U* when the electrons are n = n_D + (K U* - boundary terms) / kappa:
    more electrons than donors raise the potential energy (Eq. 9 with U = -e Phi)."""
    N, A, cx, cy, kappa = 5, 4, 1.0, 0.5, 0.2
    rng = np.random.default_rng(3)
    U = rng.normal(size=(N, A))
    nD = rng.random((N, A)) + 3.0
    Kb = O.poisson_residual(U, None, None, cx, cy, 0.1, -0.1, 0.0)
    n = nD + Kb / kappa
    assert np.abs(O.poisson_residual(U, n, nD, cx, cy, 0.1, -0.1, kappa)).max() < 1e-12
    # raising n at one atom lowers the residual there by kappa per electron
    n2 = n.copy()
    n2[2, 1] += 1.0
    F = O.poisson_residual(U, n2, nD, cx, cy, 0.1, -0.1, kappa)
    assert abs(F[2, 1] + kappa) < 1e-12 and np.abs(np.delete(F.ravel(), 2 * A + 1)).max() < 1e-12


def _poisson_device():
    dev = make_device(3, 20, 31, ge_frac=0.2)
    E = np.linspace(-1.2, 0.6, 6)
    wE = np.full(6, E[1] - E[0])
    return dev, E, wE


def test_susceptibility_matches_finite_differences():
    """chi = d n_atom / d U_atom from the dense gradient of Eqs. 1-2 equals central finite
    differences of the energy-integrated electrons per atom."""
    dev, E, wE = _poisson_device()
    N, b = 3, 20
    A = 2
    leads = [O.lead_self_energies(dev.D, dev.T, float(e), 1e-3, 0.1, -0.1, O.KT_300K) for e in E]
    U0 = np.random.default_rng(5).uniform(-0.1, 0.1, (N, A))
    chi = O.susceptibility(dev.D, dev.T, E, wE, 1e-3, U0, leads)
    h = 1e-5
    for col in (0, 3, 5):
        dU = np.zeros(N * A)
        dU[col] = h
        up = O.electrons_per_atom(dev.D, dev.T, E, wE, 1e-3, U0 + dU.reshape(N, A), leads)
        dn = O.electrons_per_atom(dev.D, dev.T, E, wE, 1e-3, U0 - dU.reshape(N, A), leads)
        fd = ((up - dn) / (2 * h)).ravel()
        assert np.abs(chi[:, col] - fd).max() < 1e-6 * max(1.0, np.abs(fd).max())


def test_poisson_newton_converges_quadratically_to_the_picard_fixed_point():
    """Newton on F(U) = 0 converges quadratically, and its U is the fixed point that a damped
    Picard iteration (solve the linear Poisson equation with the previous electrons) reaches."""
    dev, E, wE = _poisson_device()
    N, A = 3, 2
    cx, cy, kappa, eta = 1.0, 0.5, 0.05, 1e-3
    leads = [O.lead_self_energies(dev.D, dev.T, float(e), eta, 0.1, -0.1, O.KT_300K) for e in E]
    n0 = O.electrons_per_atom(dev.D, dev.T, E, wE, eta, np.zeros((N, A)), leads)
    nD = np.full((N, A), n0.mean()) + 0.2
    U, hist = O.poisson_newton(dev.D, dev.T, E, wE, eta, nD, cx, cy, 0.0, 0.0, kappa, tol=1e-11)
    assert hist[-1] < 1e-11 and len(hist) <= 8
    # quadratic: once small, each residual is far below the previous one
    big = [h for h in hist if h < 1e-2]
    for r0, r1 in zip(big, big[1:]):
        assert r1 < 10 * r0 ** 1.5
    # the Picard map's derivative kappa K^-1 chi has eigenvalues down to about -3 here, so a
    # mixing of 1/4 keeps it contracting
    K = O.poisson_matrix(N, A, cx, cy)
    Up = np.zeros((N, A))
    for _ in range(300):
        n = O.electrons_per_atom(dev.D, dev.T, E, wE, eta, Up, leads)
        rhs = (kappa * (n - nD)).ravel()   # contacts grounded: no boundary terms
        Up = 0.75 * Up + 0.25 * np.linalg.solve(K, rhs).reshape(N, A)
    assert np.abs(Up - U).max() < 1e-9
    assert np.abs(U).max() > 1e-3   # a non-trivial potential


# ---- non-uniform energy meshes -----------------------------------------------------------------

def test_scba_on_a_uniform_mesh_equals_the_index_shift_form():
    """On a uniform mesh with hbar omega a whole number of steps the interpolated Born update is
    the index-shifted one of Eqs. 4-6 (reading: E +- hbar omega, off-grid energies contribute 0)."""
    rng = np.random.default_rng(21)
    n_k, n_E, n_orb, sh = 2, 40, 5, 6
    dGR = rng.normal(size=(n_k, n_E, n_orb)) + 1j * rng.normal(size=(n_k, n_E, n_orb))
    dGL = 1j * rng.random((n_k, n_E, n_orb))
    wk = np.array([0.3, 0.7])
    dE = 0.0078125                      # a power of two: E_j + s dE lands on mesh points exactly
    E = -0.25 + dE * np.arange(n_E)
    a = O.scba_selfenergy(dGR, dGL, wk, 0.01, 0.02, sh, 0.11)
    b = O.scba_selfenergy_mesh(dGR, dGL, wk, E, 0.01, 0.02, sh * dE, 0.11)
    assert np.abs(a[0] - b[0]).max() < 1e-15 and np.abs(a[1] - b[1]).max() < 1e-15


def test_scba_mesh_interpolation_is_exact_for_linear_diag_g():
    """diag G linear in E on a random non-uniform mesh: the optical terms equal the line at
    E +- hbar omega wherever that lies on the mesh, and vanish off it."""
    rng = np.random.default_rng(22)
    E = np.sort(rng.uniform(-1.0, 1.0, 30))
    slope = rng.normal(size=3) + 1j * rng.normal(size=3)
    icpt = rng.normal(size=3) + 1j * rng.normal(size=3)
    line = lambda e: icpt + slope * e
    dG = np.array([[line(e) for e in E]])          # one k-point, weight 1
    hw = 0.137
    sR, sL = O.scba_selfenergy_mesh(dG, dG, np.ones(1), E, 0.0, 1.0, hw, 0.25)
    for j, e in enumerate(E):
        up = line(e + hw) if e + hw <= E[-1] else 0.0
        dn = line(e - hw) if e - hw >= E[0] else 0.0
        assert np.allclose(sL[j], 1.25 * up + 0.25 * dn, atol=1e-13)
        assert np.allclose(sR[j], 1.25 * dn + 0.25 * up + 0.5 * dn - 0.5 * up, atol=1e-13)


def test_trapezoid_weights_integrate_lines_exactly_on_any_mesh():
    rng = np.random.default_rng(23)
    E = np.sort(rng.uniform(-2.0, 3.0, 17))
    w = O.trapezoid_weights(E)
    assert abs(w.sum() - (E[-1] - E[0])) < 1e-14
    assert abs((w * (2.0 * E + 1.0)).sum() - ((E[-1] ** 2 + E[-1]) - (E[0] ** 2 + E[0]))) < 1e-13


def _decimate(h, alpha, z, perturb_at=0, rel=1e-14, seed=0, max_iter=100, tol=1e-13):
    """The decimation of oracle.sancho_rubio with g perturbed by rel * max|g| (complex Gaussian)
    at one doubling step; returns the surface Green's function and the steps run."""
    rng = np.random.default_rng(seed)
    b = h.shape[0]
    I = np.eye(b)
    eps_s, eps = h.astype(complex).copy(), h.astype(complex).copy()
    a, be = alpha.astype(complex).copy(), alpha.conj().T.astype(complex).copy()
    scale = max(np.abs(h).max(), np.abs(alpha).max())
    for it in range(1, max_iter + 1):
        g = np.linalg.inv(z * I - eps)
        if it == perturb_at:
            g = g + rel * np.abs(g).max() * (rng.standard_normal(g.shape)
                                             + 1j * rng.standard_normal(g.shape))
        agb, bga = a @ g @ be, be @ g @ a
        eps_s, eps = eps_s + agb, eps + agb + bga
        a, be = a @ g @ a, be @ g @ be
        if max(np.abs(a).max(), np.abs(be).max()) < tol * scale:
            break
    return np.linalg.inv(z * I - eps_s), it


def test_late_decimation_steps_barely_propagate_rounding():
    """The premise of the mixed form's lead precision schedule (fewer bits in later doubling
    steps): on a device other than the one the schedule was measured on, a 1e-14 perturbation of
    g at any step from the 15th on moves Sigma by far less than the 1e-6 accuracy target, while
    the unperturbed loop is the oracle's decimation."""
    dev = make_device(6, 12, 5151, ge_frac=0.2)
    h, t = dev.D[-1], dev.T[-1]
    worst_late = 0.0
    for E in (-1.9, -0.7, -0.05, 0.4, 1.3, 2.2):
        z = E + 1e-6j
        g0, n = _decimate(h, t, z)
        ref, n_ref, ok = O.sancho_rubio(h, t, z)
        assert ok and n == n_ref and np.abs(g0 - ref).max() <= 1e-12 * np.abs(ref).max()
        s0 = t @ g0 @ t.conj().T
        for step in range(15, n + 1):
            g1, _ = _decimate(h, t, z, perturb_at=step, seed=step)
            s1 = t @ g1 @ t.conj().T
            worst_late = max(worst_late, np.abs(s1 - s0).max() / np.abs(s0).max())
    assert worst_late < 1e-9


def test_decimation_keeps_the_interface_support():
    """The premise of the interface-coupling decimation: with a hopping supported on its last r
    rows R and first c columns C, every doubling step keeps alpha_n on C x R and beta_n on
    R x C for the left lead (alpha_0 = tau^H), and the surface self-energy lives on C x C."""
    N, b, r, c = 4, 10, 3, 4
    dev = make_device(N, b, 808, iface=(r, c))
    t = dev.T[0]
    assert np.all(t[:b - r, :] == 0) and np.all(t[:, c:] == 0)
    R, C = np.arange(b - r, b), np.arange(c)
    h = dev.D[0]
    z = 0.3 + 1e-6j
    I = np.eye(b)
    eps_s, eps = h.astype(complex).copy(), h.astype(complex).copy()
    a, be = t.conj().T.astype(complex), t.astype(complex)
    outside_a = np.ones((b, b), bool)
    outside_a[np.ix_(C, R)] = False
    for _ in range(12):
        g = np.linalg.inv(z * I - eps)
        agb, bga = a @ g @ be, be @ g @ a
        eps_s, eps = eps_s + agb, eps + agb + bga
        a, be = a @ g @ a, be @ g @ be
        assert np.all(a[outside_a] == 0) and np.all(be[outside_a.T] == 0)
    sig = O.lead_self_energies(dev.D, dev.T, 0.3, 1e-6, 0.1, -0.1, KT)["sigL"]
    assert np.all(sig[c:, :] == 0) and np.all(sig[:, c:] == 0)
