"""CPU oracle for the NEGF / recursive Green's function hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the CUDA library imports, links or calls this module; only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` use it.

Everything is plain numpy in complex128 (float64 for real quantities), written for a reader to
check against the paper by eye; library primitives used as steps: ``numpy.linalg.inv`` and ``@``.

Conventions (paper, Eqs. 1-8, "Overview"/"Claims" sections):
  * the device Hamiltonian is block tridiagonal with N slabs of b orbitals; ``Hd[i]`` = H_ii and
    ``Hu[i]`` = H_{i,i+1} (0-based), H_{i+1,i} = Hu[i]^H;
  * z = E + i*eta; the on-site potential V (eV, per orbital, ``[N, b]``) enters Eq. (1) as
    H_ii + diag(V_i) (the e*Phi term);
  * scattering self-energies of Eqs. (4)-(6) are orbital-diagonal: ``sR[i]``/``sL[i]`` are ``[b]``
    complex vectors for slab i (the paper's "diag G"), or block-diagonal with one A x A block
    per atom, given as a ``[b, b]`` matrix per slab (``atom_block_matrix``); the Born update is
    the same linear map applied to every entry of diag G or of its atom blocks;
  * leads are semi-infinite periodic copies of the end slabs (left: cell H_11, hopping H_12;
    right: cell H_NN, hopping H_{N-1,N}); Sigma^< = i f Gamma with Gamma = i(Sigma - Sigma^H);
  * density per orbital and energy  n_j(E) = Im G^<_jj / (2 pi)            (Eq. 7 integrand),
    bond current                      j_i(E) = 2 Re Tr[H_{i,i+1} G^<_{i+1,i}] (Eq. 8, read as the
    current through the bond between slabs i and i+1, in units of 1/h per spin),
    transmission (ballistic)          T(E) = Tr[Gamma_R A_NN] - Tr[Gamma_R G_NN Gamma_R G_NN^H].

Pins for every function live in ``tests/test_oracle_*.py`` (dense inversion, closed forms of the
1D chain, channel counting, current conservation, fluctuation-dissipation, finite differences).
"""
from __future__ import annotations

import numpy as np

KT_300K = 0.025852  # eV, k_B * 300 K


# ----------------------------------------------------------------------------------------------
# Occupations
# ----------------------------------------------------------------------------------------------
def fermi(E, mu, kT):
    """Fermi-Dirac occupation of the contacts (numerically stable form)."""
    x = (np.asarray(E, dtype=np.float64) - mu) / kT
    return 0.5 * (1.0 - np.tanh(0.5 * x))


def bose(hw, kT):
    """Bose occupation n0 = 1 / (exp(hw / kT) - 1) of the optical phonon (Eqs. 5-6)."""
    return 1.0 / np.expm1(hw / kT)


# ----------------------------------------------------------------------------------------------
# Lead self-energies (Eq. 3, Sigma_lead): Sancho-Rubio decimation
# ----------------------------------------------------------------------------------------------
def sancho_rubio(h, alpha, z, tol=1e-13, max_iter=100):
    """Surface Green's function of a semi-infinite periodic lead by decimation.

    Published method: Lopez Sancho, Lopez Sancho & Rubio, J. Phys. F 15, 851 (1985).  The lead's
    surface cell has on-site block ``h`` and couples to the next cell deeper into the lead through
    ``alpha`` (= H_{s,s+1}); the reverse coupling is beta = alpha^H.  Each step folds every second
    cell away:
        g   = (z - eps)^-1
        eps_s <- eps_s + alpha g beta
        eps   <- eps + alpha g beta + beta g alpha
        alpha <- alpha g alpha,  beta <- beta g beta
    and stops once max(|alpha|_max, |beta|_max) < tol * max(|h|_max, |alpha_0|_max).
    Returns (g_s = (z - eps_s)^-1, iterations, converged).
    """
    b = h.shape[0]
    I = np.eye(b)
    eps_s = h.astype(np.complex128).copy()
    eps = h.astype(np.complex128).copy()
    a = alpha.astype(np.complex128).copy()
    be = alpha.conj().T.astype(np.complex128).copy()
    scale = max(np.abs(h).max(), np.abs(alpha).max(), 1e-300)
    it = 0
    converged = False
    for it in range(1, max_iter + 1):
        g = np.linalg.inv(z * I - eps)
        agb = a @ g @ be
        bga = be @ g @ a
        eps_s = eps_s + agb
        eps = eps + agb + bga
        a = a @ g @ a
        be = be @ g @ be
        if max(np.abs(a).max(), np.abs(be).max()) < tol * scale:
            converged = True
            break
    return np.linalg.inv(z * I - eps_s), it, converged


def lead_self_energies(Hd, Hu, E, eta, mu_L, mu_R, kT, tol=1e-13, max_iter=100):
    """Retarded and lesser lead self-energies of both contacts at one energy.

    Left lead: surface cell H_11 coupled deeper into the lead by alpha_L = H_12^H; the device's
    slab 1 sees Sigma_L = H_12^H g_L H_12.  Right lead: surface cell H_NN coupled deeper by
    alpha_R = H_{N-1,N}; slab N sees Sigma_R = H_{N-1,N} g_R H_{N-1,N}^H.
    Gamma = i (Sigma - Sigma^H) and Sigma^< = i f(E) Gamma with each contact's Fermi level.
    For N == 1 there is no device hopping to copy, so both leads are flat (Sigma = 0).
    """
    z = E + 1j * eta
    b = Hd.shape[1]
    N = Hd.shape[0]
    if N < 2:
        Z = np.zeros((b, b), dtype=np.complex128)
        return dict(sigL=Z, sigR=Z.copy(), gamL=Z.copy(), gamR=Z.copy(), lesL=Z.copy(),
                    lesR=Z.copy(), itL=0, itR=0, convL=True, convR=True)
    tauL = Hu[0]
    tauR = Hu[N - 2]
    gL, itL, cL = sancho_rubio(Hd[0], tauL.conj().T, z, tol, max_iter)
    gR, itR, cR = sancho_rubio(Hd[N - 1], tauR, z, tol, max_iter)
    sigL = tauL.conj().T @ gL @ tauL
    sigR = tauR @ gR @ tauR.conj().T
    gamL = 1j * (sigL - sigL.conj().T)
    gamR = 1j * (sigR - sigR.conj().T)
    fL = float(fermi(E, mu_L, kT))
    fR = float(fermi(E, mu_R, kT))
    return dict(sigL=sigL, sigR=sigR, gamL=gamL, gamR=gamR, lesL=1j * fL * gamL,
                lesR=1j * fR * gamR, itL=itL, itR=itR, convL=cL, convR=cR, gL=gL, gR=gR)


# ----------------------------------------------------------------------------------------------
# Eqs. (1)-(2) by their plain definition (dense inversion; tiny devices only)
# ----------------------------------------------------------------------------------------------
def assemble_dense(Hd, Hu):
    N, b = Hd.shape[0], Hd.shape[1]
    H = np.zeros((N * b, N * b), dtype=np.complex128)
    for i in range(N):
        H[i * b:(i + 1) * b, i * b:(i + 1) * b] = Hd[i]
    for i in range(N - 1):
        H[i * b:(i + 1) * b, (i + 1) * b:(i + 2) * b] = Hu[i]
        H[(i + 1) * b:(i + 2) * b, i * b:(i + 1) * b] = Hu[i].conj().T
    return H


def dense_self_energies(N, b, leads, sR=None, sL=None):
    """Full (N b)^2 Sigma^R and Sigma^< of Eq. (3): leads on the end slabs plus diagonal scattering."""
    SR = np.zeros((N * b, N * b), dtype=np.complex128)
    SL = np.zeros_like(SR)
    SR[:b, :b] += leads["sigL"]
    SL[:b, :b] += leads["lesL"]
    SR[(N - 1) * b:, (N - 1) * b:] += leads["sigR"]
    SL[(N - 1) * b:, (N - 1) * b:] += leads["lesR"]
    for S, X in ((SR, sR), (SL, sL)):
        if X is None:
            continue
        X = np.asarray(X)
        if X.ndim == 3:  # one b x b matrix per slab (block-diagonal scattering)
            for i in range(N):
                S[i * b:(i + 1) * b, i * b:(i + 1) * b] += X[i]
        else:
            S[np.diag_indices(N * b)] += X.reshape(-1)
    return SR, SL


def dense_green(Hd, Hu, E, eta, V, leads, sR=None, sL=None):
    """G^R = (z - H - V - Sigma^R)^-1 (Eq. 1) and G^< = G^R Sigma^< G^R^H (Eq. 2), dense."""
    N, b = Hd.shape[0], Hd.shape[1]
    H = assemble_dense(Hd, Hu)
    if V is not None:
        H = H + np.diag(np.asarray(V, dtype=np.float64).reshape(-1))
    SR, SL = dense_self_energies(N, b, leads, sR, sL)
    G = np.linalg.inv((E + 1j * eta) * np.eye(N * b) - H - SR)
    GL = G @ SL @ G.conj().T
    return G, GL


# ----------------------------------------------------------------------------------------------
# Recursive Green's function (exact diagonal / first off-diagonal blocks of Eqs. 1-2)
# ----------------------------------------------------------------------------------------------
def rgf(Hd, Hu, E, eta, V, leads, sR=None, sL=None):
    """Forward sweep of left-connected g, g^<, then backward sweep for the full blocks.

    Forward (i = 1..N):
        g_i   = (z - H_ii - V_i - Sigma_i - t_{i-1}^H g_{i-1} t_{i-1})^-1
        g^<_i = g_i (Sigma^<_i + t_{i-1}^H g^<_{i-1} t_{i-1}) g_i^H
    where t_i = H_{i,i+1}, Sigma_i holds the scattering self-energy of slab i plus Sigma_L (slab 1)
    and Sigma_R (slab N).
    Backward (i = N-1..1), with L = g_i t_i:
        G_{i,i+1}   = L G_{i+1}
        G_ii        = g_i + G_{i,i+1} t_i^H g_i
        X           = G_{i,i+1} t_i^H g^<_i
        G^<_ii      = g^<_i + L G^<_{i+1} L^H + X - X^H
        G^<_{i+1,i} = G_{i+1} t_i^H g^<_i + G^<_{i+1} L^H
    Returns dict(G=[G_ii], GL=[G^<_ii], GLoff=[G^<_{i+1,i}], g=[g_i], gl=[g^<_i]).
    """
    N, b = Hd.shape[0], Hd.shape[1]
    z = E + 1j * eta
    I = np.eye(b)
    g = [None] * N
    gl = [None] * N
    for i in range(N):
        M = z * I - Hd[i]
        S = np.zeros((b, b), dtype=np.complex128)
        if V is not None:
            M = M - np.diag(np.asarray(V[i], dtype=np.float64))
        # scattering self-energy of slab i: a diagonal (vector) or a b x b matrix
        if sR is not None:
            M = M - (sR[i] if np.ndim(sR[i]) == 2 else np.diag(sR[i]))
        if sL is not None:
            S = S + (sL[i] if np.ndim(sL[i]) == 2 else np.diag(sL[i]))
        if i == 0:
            M = M - leads["sigL"]
            S = S + leads["lesL"]
        if i == N - 1:
            M = M - leads["sigR"]
            S = S + leads["lesR"]
        if i > 0:
            t = Hu[i - 1]
            M = M - t.conj().T @ g[i - 1] @ t
            S = S + t.conj().T @ gl[i - 1] @ t
        g[i] = np.linalg.inv(M)
        gl[i] = g[i] @ S @ g[i].conj().T
    G = [None] * N
    GL = [None] * N
    GLoff = [None] * max(N - 1, 0)
    G[N - 1] = g[N - 1]
    GL[N - 1] = gl[N - 1]
    for i in range(N - 2, -1, -1):
        t = Hu[i]
        L = g[i] @ t
        Gi_ip1 = L @ G[i + 1]
        G[i] = g[i] + Gi_ip1 @ t.conj().T @ g[i]
        X = Gi_ip1 @ t.conj().T @ gl[i]
        GL[i] = gl[i] + L @ GL[i + 1] @ L.conj().T + X - X.conj().T
        GLoff[i] = G[i + 1] @ t.conj().T @ gl[i] + GL[i + 1] @ L.conj().T
    return dict(G=G, GL=GL, GLoff=GLoff, g=g, gl=gl)


# ----------------------------------------------------------------------------------------------
# Observables (Eqs. 7-8 integrands, transmission)
# ----------------------------------------------------------------------------------------------
def atom_blocks(X, A):
    """The A x A diagonal blocks of a b x b matrix X as a row of b A entries: entry (r, c), r and
    c in the same atom (orbitals [A a, A a + A)), at r A + (c mod A)."""
    b = X.shape[0]
    out = np.zeros(b * A, dtype=np.complex128)
    for r in range(b):
        a0 = (r // A) * A
        for c in range(a0, a0 + A):
            out[r * A + (c - a0)] = X[r, c]
    return out


def atom_block_matrix(row, b, A):
    """Inverse of atom_blocks: the b x b block-diagonal matrix with the A x A blocks of `row`."""
    X = np.zeros((b, b), dtype=np.complex128)
    for r in range(b):
        a0 = (r // A) * A
        for c in range(a0, a0 + A):
            X[r, c] = row[r * A + (c - a0)]
    return X


def density_from_blocks(GL):
    """n_j(E) = Im G^<_jj / (2 pi) for every orbital, slab-major ``[N*b]``."""
    return np.concatenate([np.imag(np.diag(x)) for x in GL]) / (2.0 * np.pi)


def current_from_blocks(Hu, GLoff):
    """j_i(E) = 2 Re Tr[H_{i,i+1} G^<_{i+1,i}] for the N-1 bonds."""
    return np.array([2.0 * np.real(np.trace(Hu[i] @ GLoff[i])) for i in range(len(GLoff))])


def transmission_from_GNN(G_NN, gamR):
    """T = Tr[Gamma_R A_NN] - Tr[Gamma_R G_NN Gamma_R G_NN^H], A = i (G - G^H)."""
    A = 1j * (G_NN - G_NN.conj().T)
    return float(np.real(np.trace(gamR @ A) - np.trace(gamR @ G_NN @ gamR @ G_NN.conj().T)))


def transmission_caroli_dense(G, gamL, gamR, N, b):
    """Caroli formula Tr[Gamma_L G_1N Gamma_R G_1N^H] from a dense G (cross-check)."""
    G1N = G[:b, (N - 1) * b:]
    return float(np.real(np.trace(gamL @ G1N @ gamR @ G1N.conj().T)))


def solve_point(Hd, Hu, E, eta, V=None, *, eta_lead=None, mu_L=0.1, mu_R=-0.1, kT=KT_300K,
                sR=None, sL=None, leads=None, sr_tol=1e-13, sr_max_iter=100):
    """Leads + RGF + observables at one (E, k) point; returns a dict of FP64 results."""
    if leads is None:
        leads = lead_self_energies(Hd, Hu, E, eta if eta_lead is None else eta_lead, mu_L, mu_R,
                                   kT, sr_tol, sr_max_iter)
    r = rgf(Hd, Hu, E, eta, V, leads, sR, sL)
    N = Hd.shape[0]
    out = dict(
        density=density_from_blocks(r["GL"]),
        current=current_from_blocks(Hu, r["GLoff"]),
        transmission=transmission_from_GNN(r["G"][N - 1], leads["gamR"]),
        diagGR=np.concatenate([np.diag(x) for x in r["G"]]),
        diagGL=np.concatenate([np.diag(x) for x in r["GL"]]),
        leads=leads, blocks=r,
    )
    return out


def integrate(values, weights):
    """Sum_p w_p values[p] in FP64, in point order (the E / k quadrature of Eqs. 7-8)."""
    values = np.asarray(values, dtype=np.float64)
    weights = np.asarray(weights, dtype=np.float64)
    acc = np.zeros(values.shape[1:], dtype=np.float64)
    for p in range(values.shape[0]):
        acc = acc + weights[p] * values[p]
    return acc


# ----------------------------------------------------------------------------------------------
# Self-consistent Born step, Eqs. (4)-(6)
# ----------------------------------------------------------------------------------------------
def scba_selfenergy(dGR, dGL, wk, D_ac, D_op, shift, n0):
    """Orbital-diagonal phonon self-energies from diag G over all (k', E).

    dGR, dGL: ``[n_k, n_E, n_orb]`` complex diagonals of G^R, G^<.  wk: k' weights (the integral
    over k' of Eqs. 4-6 becomes sum_k' w_k'), so the result is the same for every k.
    Acoustic (Eq. 4, elastic):   Sigma_ac^{R,<}(E) = D_ac * sum_k' w dG^{R,<}(k', E)
    Optical  (Eq. 5):            Sigma_op^<(E) = D_op * sum_k' w [(1+n0) dG^<(E+hw) + n0 dG^<(E-hw)]
    Optical  (Eq. 6):            Sigma_op^R(E) = D_op * sum_k' w [(1+n0) dG^R(E-hw) + n0 dG^R(E+hw)
                                                 + 0.5 dG^<(E-hw) - 0.5 dG^<(E+hw)]
    hw is ``shift`` grid steps; energies shifted off the grid contribute zero.
    Returns (Sigma^R, Sigma^<), each ``[n_E, n_orb]``.
    """
    dGR = np.asarray(dGR, dtype=np.complex128)
    dGL = np.asarray(dGL, dtype=np.complex128)
    n_k, n_E, n_orb = dGR.shape
    sumR = np.zeros((n_E, n_orb), dtype=np.complex128)
    sumL = np.zeros((n_E, n_orb), dtype=np.complex128)
    for k in range(n_k):
        sumR = sumR + wk[k] * dGR[k]
        sumL = sumL + wk[k] * dGL[k]

    def at(arr, j):
        if 0 <= j < n_E:
            return arr[j]
        return np.zeros(n_orb, dtype=np.complex128)

    sigR = np.zeros((n_E, n_orb), dtype=np.complex128)
    sigL = np.zeros((n_E, n_orb), dtype=np.complex128)
    for j in range(n_E):
        up, dn = j + shift, j - shift
        sigR[j] = D_ac * sumR[j] + D_op * ((1.0 + n0) * at(sumR, dn) + n0 * at(sumR, up)
                                           + 0.5 * at(sumL, dn) - 0.5 * at(sumL, up))
        sigL[j] = D_ac * sumL[j] + D_op * ((1.0 + n0) * at(sumL, up) + n0 * at(sumL, dn))
    return sigR, sigL


def scba_step(dGR, dGL, wk, D_ac, D_op, shift, n0, sig_old_R, sig_old_L, mix=1.0):
    """One Born update with linear mixing; returns (Sigma^R, Sigma^<, max |Delta Sigma|)."""
    nR, nL = scba_selfenergy(dGR, dGL, wk, D_ac, D_op, shift, n0)
    newR = (1.0 - mix) * sig_old_R + mix * nR
    newL = (1.0 - mix) * sig_old_L + mix * nL
    delta = max(np.abs(newR - sig_old_R).max(), np.abs(newL - sig_old_L).max())
    return newR, newL, float(delta)


def interp_on_mesh(values, E, x):
    """Linear interpolation of values[j] (rows over the sorted mesh E) at energy x; zero when x
    lies outside [E[0], E[-1]]."""
    E = np.asarray(E, dtype=np.float64)
    if x < E[0] or x > E[-1]:
        return np.zeros_like(values[0])
    m = int(np.searchsorted(E, x, side="right")) - 1
    if m >= len(E) - 1:
        return values[len(E) - 1].copy()
    t = (x - E[m]) / (E[m + 1] - E[m])
    return (1.0 - t) * values[m] + t * values[m + 1]


def scba_selfenergy_mesh(dGR, dGL, wk, E, D_ac, D_op, hw, n0):
    """Eqs. (4)-(6) on a non-uniform energy mesh E: as scba_selfenergy, with diag G at E +- hw
    taken by linear interpolation between the mesh points around it (zero off the mesh)."""
    dGR = np.asarray(dGR, dtype=np.complex128)
    dGL = np.asarray(dGL, dtype=np.complex128)
    n_k, n_E, n_orb = dGR.shape
    sumR = np.zeros((n_E, n_orb), dtype=np.complex128)
    sumL = np.zeros((n_E, n_orb), dtype=np.complex128)
    for k in range(n_k):
        sumR = sumR + wk[k] * dGR[k]
        sumL = sumL + wk[k] * dGL[k]
    sigR = np.zeros((n_E, n_orb), dtype=np.complex128)
    sigL = np.zeros((n_E, n_orb), dtype=np.complex128)
    for j in range(n_E):
        up, dn = E[j] + hw, E[j] - hw
        sigR[j] = D_ac * sumR[j] + D_op * ((1.0 + n0) * interp_on_mesh(sumR, E, dn)
                                           + n0 * interp_on_mesh(sumR, E, up)
                                           + 0.5 * interp_on_mesh(sumL, E, dn)
                                           - 0.5 * interp_on_mesh(sumL, E, up))
        sigL[j] = D_ac * sumL[j] + D_op * ((1.0 + n0) * interp_on_mesh(sumL, E, up)
                                           + n0 * interp_on_mesh(sumL, E, dn))
    return sigR, sigL


def scba_step_mesh(dGR, dGL, wk, E, D_ac, D_op, hw, n0, sig_old_R, sig_old_L, mix=1.0):
    """One Born update on a non-uniform mesh with linear mixing."""
    nR, nL = scba_selfenergy_mesh(dGR, dGL, wk, E, D_ac, D_op, hw, n0)
    newR = (1.0 - mix) * sig_old_R + mix * nR
    newL = (1.0 - mix) * sig_old_L + mix * nL
    delta = max(np.abs(newR - sig_old_R).max(), np.abs(newL - sig_old_L).max())
    return newR, newL, float(delta)


def trapezoid_weights(E):
    """Trapezoid weights of a sorted, possibly non-uniform energy mesh."""
    E = np.asarray(E, dtype=np.float64)
    w = np.zeros(len(E))
    for j in range(len(E) - 1):
        h = E[j + 1] - E[j]
        w[j] += 0.5 * h
        w[j + 1] += 0.5 * h
    return w


# ----------------------------------------------------------------------------------------------
# Gradient of the observables with respect to the on-site potential (dense definition)
# ----------------------------------------------------------------------------------------------
def omega_dense(Hu, N, b, c, d):
    """Omega such that Re Tr[Omega G^<] = sum_j c_j n_j(E) + sum_i d_i j_i(E)."""
    Om = np.zeros((N * b, N * b), dtype=np.complex128)
    if c is not None:
        Om[np.diag_indices(N * b)] += -1j * np.asarray(c, dtype=np.float64).reshape(-1) / (2 * np.pi)
    if d is not None:
        for i in range(N - 1):
            Om[i * b:(i + 1) * b, (i + 1) * b:(i + 2) * b] += 2.0 * d[i] * Hu[i]
    return Om


def gradient_dense(Hd, Hu, E, eta, V, leads, c, d, sR=None, sL=None):
    """dL/dV_q for L = sum_j c_j n_j(E) + sum_i d_i j_i(E), by differentiating Eqs. (1)-(2).

    With M = z - H - V - Sigma, dG/dV_q = G P_q G and dG^</dV_q = G P_q G^< + G^< P_q G^H
    (P_q the projector on orbital q; Sigma does not depend on V), so with L = Re Tr[Omega G^<]:
        dL/dV_q = Re[(G^< Omega G)_qq + (G^H Omega G^<)_qq].
    Returns ``[N, b]``.
    """
    N, b = Hd.shape[0], Hd.shape[1]
    G, GL = dense_green(Hd, Hu, E, eta, V, leads, sR, sL)
    Om = omega_dense(Hu, N, b, c, d)
    grad = np.real(np.diag(GL @ Om @ G) + np.diag(G.conj().T @ Om @ GL))
    return grad.reshape(N, b)


# ----------------------------------------------------------------------------------------------
# NEGF-Poisson self-consistency, Eq. (9)
# ----------------------------------------------------------------------------------------------
ORBITALS_PER_ATOM = 10


def atom_sums(orb, N, b, per=ORBITALS_PER_ATOM):
    """Electrons per atom from a per-orbital array [N*b]: atom a of slab i owns orbitals
    per*a .. per*a + per - 1 of that slab.  Returns [N, A]."""
    orb = np.asarray(orb, dtype=np.float64).reshape(N, b)
    A = -(-b // per)
    out = np.zeros((N, A))
    for i in range(N):
        for a in range(A):
            out[i, a] = orb[i, per * a:min(per * a + per, b)].sum()
    return out


def atom_to_orbitals(U, b, per=ORBITALS_PER_ATOM):
    """Per-orbital potential [N, b] from one value per atom [N, A]."""
    U = np.asarray(U, dtype=np.float64)
    N = U.shape[0]
    out = np.zeros((N, b))
    for i in range(N):
        for o in range(b):
            out[i, o] = U[i, o // per]
    return out


def poisson_residual(U, n, n_D, cx, cy, UL, UR, kappa):
    """Eq. (9) for the potential energy U = -e Phi on the atom grid, as a residual:

        F[i,a] = cx (2 U[i,a] - U[i-1,a] - U[i+1,a]) + cy (2 U[i,a] - U[i,a-1] - U[i,a+1])
                 - kappa (n[i,a] - n_D[i,a])

    (finite differences of -div(eps grad U); slab i along transport with the contacts held at
    U[-1,:] = UL and U[N,:] = UR, atom a periodic across the slab; n = None: operator only).
    """
    U = np.asarray(U, dtype=np.float64)
    N, A = U.shape
    F = np.zeros((N, A))
    for i in range(N):
        for a in range(A):
            left = U[i - 1, a] if i > 0 else UL
            right = U[i + 1, a] if i < N - 1 else UR
            r = cx * (2 * U[i, a] - left - right)
            if A > 1:
                r += cy * (2 * U[i, a] - U[i, (a - 1) % A] - U[i, (a + 1) % A])
            if n is not None:
                r -= kappa * (n[i, a] - (0.0 if n_D is None else n_D[i, a]))
            F[i, a] = r
    return F


def poisson_matrix(N, A, cx, cy):
    """The linear part of poisson_residual as a matrix K over the flattened (i, a) grid (the
    residual of a unit potential at one atom with grounded contacts)."""
    K = np.zeros((N * A, N * A))
    for j in range(N * A):
        e = np.zeros(N * A)
        e[j] = 1.0
        K[:, j] = poisson_residual(e.reshape(N, A), None, None, cx, cy, 0.0, 0.0, 0.0).ravel()
    return K


def electrons_per_atom(Hd, Hu, E, wE, eta, U, leads, per=ORBITALS_PER_ATOM):
    """n = sum_E w_E n(E) per atom (Eq. 7) with the potential U [N, A] in Eq. (1)."""
    N, b = Hd.shape[0], Hd.shape[1]
    V = atom_to_orbitals(U, b, per)
    dens = [solve_point(Hd, Hu, float(e), eta, V, leads=lo)["density"]
            for e, lo in zip(E, leads)]
    return atom_sums(integrate(dens, wE), N, b, per)


def susceptibility(Hd, Hu, E, wE, eta, U, leads, per=ORBITALS_PER_ATOM):
    """chi[a, a'] = d n_a / d U_a' (n_a energy-integrated), one row per atom from the dense
    definition of the gradient (gradient_dense with the cotangent on atom a's orbitals)."""
    N, b = Hd.shape[0], Hd.shape[1]
    A = -(-b // per)
    V = atom_to_orbitals(U, b, per)
    chi = np.zeros((N * A, N * A))
    for i in range(N):
        for a in range(A):
            c = np.zeros((N, b))
            c[i, per * a:min(per * a + per, b)] = 1.0
            g = np.zeros((N, b))
            for e, w, lo in zip(E, wE, leads):
                g += w * gradient_dense(Hd, Hu, float(e), eta, V, lo, c, None)
            chi[i * A + a] = atom_sums(g.ravel(), N, b, per).ravel()
    return chi


def poisson_newton(Hd, Hu, E, wE, eta, n_D, cx, cy, UL, UR, kappa, U0=None, tol=1e-9,
                   max_iter=30, mu_L=0.1, mu_R=-0.1, kT=KT_300K, per=ORBITALS_PER_ATOM):
    """Self-consistent solution of Eqs. (1), (7) and (9): Newton's method on F(U) = 0 with
    F = poisson_residual(U, n(U), ...) and the Jacobian J = K - kappa chi.  Lead self-energies
    do not depend on U and are computed once per energy.  Returns (U, list of max |F|)."""
    N, b = Hd.shape[0], Hd.shape[1]
    A = -(-b // per)
    leads = [lead_self_energies(Hd, Hu, float(e), eta, mu_L, mu_R, kT) for e in E]
    U = np.zeros((N, A)) if U0 is None else np.array(U0, dtype=np.float64)
    K = poisson_matrix(N, A, cx, cy)
    hist = []
    for _ in range(max_iter):
        n = electrons_per_atom(Hd, Hu, E, wE, eta, U, leads, per)
        F = poisson_residual(U, n, n_D, cx, cy, UL, UR, kappa)
        hist.append(float(np.abs(F).max()))
        if hist[-1] < tol:
            break
        J = K - kappa * susceptibility(Hd, Hu, E, wE, eta, U, leads, per)
        U = U + np.linalg.solve(J, -F.ravel()).reshape(N, A)
    return U, hist
