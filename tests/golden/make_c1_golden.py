"""Writes c1_oracle.json: oracle values of the benchmark device (N = 70 slabs x 400 x 400 blocks).

The paper prints no worked example, so these stored values come from the CPU oracle alone (pinned
by tests/test_oracle_pins.py against dense inversion, closed forms and conservation laws).  This
script calls only ``oracle`` and the seeded input generator ``workloads``; nothing here comes
from the CUDA path.

Workload: the alloy device of the throughput benchmark -- N = 70 slabs, b = 400 orbitals
(40 atoms x 10), p(Ge) = 0.1, seed 1001, transverse k-points k_m = -pi + 2 pi (m + 1/2) / 8 with
k-independent hoppings, 512 energies linspace(-3, 3) with trapezoid weights, eta = 1e-6 in leads
and device, contacts mu_L = +0.1 eV, mu_R = -0.1 eV at 300 K.

Stored:
  * the whole k-slice m = 2 (k = -3 pi / 8): T(E) at all 512 energies and the energy integrals
    (trapezoid weights) of the per-atom density (sum of each atom's 10 orbitals of Eq. 7's
    integrand) and of the bond currents (Eq. 8 read as 2 Re Tr[H_{i,i+1} G^<_{i+1,i}]);
  * per-point values -- per-slab density sums, bond currents, T -- at the energies of that slice
    chosen by select() (16 evenly spaced, the 12 nearest the bias window, 8 at each edge of the
    transmitting band -- on this device the band covers the whole grid, so these are the grid's
    ends -- and the 4 energies 210-213; 38 distinct energies) and at 16 of them on the partner
    slice m = 5 (k = +3 pi / 8): 54 points.

    python tests/golden/make_c1_golden.py [--jobs 8]

About 530 oracle points: ~40 minutes on 8 cores.
"""
import argparse
import json
import multiprocessing as mp
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c1_oracle.json")
N, B, SEED, N_E, N_K, ETA = 70, 400, 1001, 512, 8, 1e-6
K_MAIN, K_PARTNER = 2, 5
ATOM = 10


def _hd(m):
    from workloads import make_device, hamiltonian_k, k_grid
    dev = make_device(N, B, SEED, ge_frac=0.1, with_k=True)
    ks, _ = k_grid(N_K)
    return hamiltonian_k(dev, float(ks[m]))[0], dev.T


def _init():
    try:
        from threadpoolctl import threadpool_limits
        threadpool_limits(1)
    except Exception:
        pass


def _point(args):
    m, e_idx = args
    import oracle as O
    from workloads import energy_grid_linspace
    Hd, Hu = _CACHE.setdefault(m, _hd(m))
    E, _ = energy_grid_linspace(-3.0, 3.0, N_E)
    r = O.solve_point(Hd, Hu, float(E[e_idx]), ETA, None, eta_lead=ETA)
    return (m, e_idx, r["density"], r["current"], float(r["transmission"]))


_CACHE = {}


def select(T):
    """Energy indices of the main slice: even spread, bias window, band edges, 210-213."""
    from workloads import energy_grid_linspace
    E, _ = energy_grid_linspace(-3.0, 3.0, N_E)
    sel = set(np.linspace(0, N_E - 1, 16).round().astype(int).tolist())
    sel |= set(np.argsort(np.abs(E))[:12].tolist())
    on = np.nonzero(T > 1e-3)[0]
    lo, hi = int(on[0]), int(on[-1])
    sel |= set(range(max(lo - 4, 0), lo + 4)) | set(range(hi - 3, min(hi + 5, N_E)))
    sel |= {210, 211, 212, 213}
    return sorted(sel)


def compute(jobs):
    import oracle as O
    from workloads import energy_grid_linspace
    E, wE = energy_grid_linspace(-3.0, 3.0, N_E)
    ctx = mp.get_context("spawn")
    with ctx.Pool(jobs, initializer=_init) as pool:
        main = pool.map(_point, [(K_MAIN, j) for j in range(N_E)], chunksize=4)
        T = np.array([r[4] for r in main])
        sel = select(T)
        part_sel = sel[::max(1, len(sel) // 16)][:16]
        partner = pool.map(_point, [(K_PARTNER, j) for j in part_sel], chunksize=1)
    dens = [r[2] for r in main]
    cur = [r[3] for r in main]
    atoms = O.integrate(dens, wE).reshape(N * B // ATOM, ATOM).sum(axis=1)
    jint = O.integrate(cur, wE)

    def pts(rows):
        return [dict(k_index=int(m), energy_index=int(j), E=float(E[j]),
                     slab_density=d.reshape(N, B).sum(axis=1).tolist(), current=c.tolist(),
                     transmission=t) for (m, j, d, c, t) in rows]
    return dict(
        workload=("N=70 slabs x 400x400 blocks (40 atoms x 10 orbitals), p(Ge)=0.1, seed 1001, "
                  "k_m = -pi + 2 pi (m + 1/2) / 8, 512 energies linspace(-3,3), eta=1e-6"),
        source="oracle/negf_oracle.py solve_point and integrate (tests/golden/make_c1_golden.py)",
        N=N, b=B, eta=ETA, n_E=N_E, n_k=N_K, k_main=K_MAIN, k_partner=K_PARTNER,
        transmission_main=T.tolist(),
        integrated_atom_density_main=atoms.tolist(),
        integrated_current_main=jint.tolist(),
        points=pts([main[j] for j in sel]) + pts(partner))


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=os.cpu_count() or 1)
    a = ap.parse_args()
    data = compute(a.jobs)
    with open(OUT, "w") as f:
        json.dump(data, f, separators=(",", ":"))
        f.write("\n")
    print("wrote", OUT)
