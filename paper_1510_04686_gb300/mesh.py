"""Adaptive non-uniform energy meshes for the energy integrals of Eqs. 7-8 and the Born step.

Resonances of width eta make the integrands of Eq. 7 (density) and Eq. 8 (current) sharply
peaked; a uniform mesh fine enough for the narrowest of them wastes points everywhere else.
refine_mesh bisects, round by round, the intervals of a trapezoid mesh whose midpoint test fails,
and asks for all new energies of a round in one batched evaluation, so every round is one
batched RGF solve of uneven size.  adaptive_energy_mesh runs it with the library's solve.
Host logic only: every integrand value comes from the library.
"""
from __future__ import annotations

import numpy as np


def trapezoid_weights(E):
    """Trapezoid weights of a sorted, possibly non-uniform mesh."""
    E = np.asarray(E, dtype=np.float64)
    w = np.zeros(len(E))
    h = np.diff(E)
    w[:-1] += 0.5 * h
    w[1:] += 0.5 * h
    return w


def refine_mesh(evaluate, E_lo, E_hi, n_init=33, tol=1e-4, max_points=4096, max_rounds=24):
    """Adaptive trapezoid mesh on [E_lo, E_hi].

    evaluate(E) -> array [len(E), n_features] of the integrands at the energies E (one call per
    round).  An interval [a, b] with midpoint m passes when its trapezoid-minus-midpoint
    difference, an estimate of its quadrature error,
        (b - a) * max_f |(f(a) + f(b)) / 2 - f(m)| <= tol * scale * (b - a) / (E_hi - E_lo),
    with scale = max_f |f| over the mesh so far, i.e. when its error density is below tol
    relative to the integrand's scale.  Failing intervals are bisected (their midpoint joins the
    mesh and both halves are tested in the next round); the midpoints of passing intervals join
    the mesh too.  Stops when every interval passes, or the mesh would exceed max_points, or after
    max_rounds rounds.  Returns (E, values, weights, rounds) with E sorted and trapezoid weights.
    """
    E = np.linspace(E_lo, E_hi, n_init)
    F = np.asarray(evaluate(E), dtype=np.float64).reshape(len(E), -1)
    pts = {float(e): f for e, f in zip(E, F)}
    active = list(zip(E[:-1], E[1:]))
    span = E_hi - E_lo
    rounds = 0
    while active and rounds < max_rounds and len(pts) + len(active) <= max_points:
        rounds += 1
        mids = np.array([0.5 * (a + b) for a, b in active])
        Fm = np.asarray(evaluate(mids), dtype=np.float64).reshape(len(mids), -1)
        scale = max(np.abs(np.array(list(pts.values()))).max(), np.abs(Fm).max(), 1e-300)
        nxt = []
        for (a, b), m, fm in zip(active, mids, Fm):
            err = (b - a) * np.abs(0.5 * (pts[a] + pts[b]) - fm).max()
            pts[float(m)] = fm
            if err > tol * scale * (b - a) / span:
                nxt += [(a, float(m)), (float(m), b)]
        active = nxt
    E = np.array(sorted(pts))
    F = np.array([pts[e] for e in E])
    return E, F, trapezoid_weights(E), rounds


def adaptive_energy_mesh(dev, sys_index, opt, E_lo, E_hi, n_init=33, tol=1e-4,
                         max_points=4096, max_rounds=24):
    """Adaptive mesh for one system of `dev` (the Hamiltonian sys_index): the integrands refined
    on are T(E), the electrons of every slab (Eq. 7 summed over the slab) and the bond currents
    (Eq. 8), each round solved by one batched lead + RGF call of the library.  Returns
    dict(E, w, density [n, N*b], current [n, N-1], transmission [n], rounds), host arrays, E
    sorted and w its trapezoid weights."""
    import torch

    from . import negf as _n
    N, b = dev.N, dev.b
    dv = dev.H_diag.device
    store = {}

    def evaluate(E):
        Et = torch.as_tensor(np.asarray(E, dtype=np.float64), device=dv)
        st = torch.full((len(E),), int(sys_index), dtype=torch.int32, device=dv)
        lead = _n.lead_selfenergy(dev, Et, st, opt)
        out = _n.rgf_solve(dev, Et, st, lead["sigma_R"], lead["sigma_L"], opt)
        dens = out["density"].cpu().numpy()
        cur = out["current"].cpu().numpy() if N > 1 else np.zeros((len(E), 0))
        T = out["transmission"].cpu().numpy()
        bad = (out["status"] | lead["status"]).cpu().numpy()
        if np.any(bad):
            raise _n.NegfError(6, "adaptive_energy_mesh", f"point status {bad.max()}")
        for q, e in enumerate(E):
            store[float(e)] = (dens[q], cur[q], T[q])
        return np.concatenate([T[:, None], dens.reshape(len(E), N, b).sum(axis=2), cur], axis=1)

    E, _, w, rounds = refine_mesh(evaluate, E_lo, E_hi, n_init, tol, max_points, max_rounds)
    return dict(E=E, w=w, rounds=rounds,
                density=np.array([store[float(e)][0] for e in E]),
                current=np.array([store[float(e)][1] for e in E]),
                transmission=np.array([store[float(e)][2] for e in E]))
