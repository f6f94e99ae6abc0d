"""Writes config0_oracle.json: oracle values for the small ballistic workload.

The paper prints no worked example (its figures are I-V curves and scaling plots), so the stored
values here come from the CPU oracle alone, pinned by tests/test_oracle_pins.py against dense
inversion, closed forms and conservation laws.  This script calls only ``oracle`` and the seeded
input generator ``workloads``; nothing here comes from the CUDA path.

Workload: N = 20 slabs x 40 x 40 blocks (4 atoms x 10 orbitals), seed 1000, 64 energies
linspace(-3, 3) with trapezoid weights, eta = 1e-6 in leads and device, one k-point.  Stored:
per-slab density sum_j n_j(E) (Eq. 7 integrand, summed over the slab's orbitals), bond currents
j_i(E) (Eq. 8 read as 2 Re Tr[H_{i,i+1} G^<_{i+1,i}]) and T(E) at every fourth energy, and the
energy integrals of the per-slab density and bond current over all 64 energies.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from workloads import config_workload  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "config0_oracle.json")
STRIDE = 4


def compute():
    w = config_workload(0)
    dev, E, wE, eta = w["device"], w["E"], w["wE"], w["eta"]
    N, b = dev.D.shape[0], dev.D.shape[1]
    pts = [O.solve_point(dev.D, dev.T, float(e), eta, None, eta_lead=eta) for e in E]
    slab = np.array([p["density"].reshape(N, b).sum(axis=1) for p in pts])
    cur = np.array([p["current"] for p in pts])
    T = np.array([p["transmission"] for p in pts])
    sel = np.arange(0, len(E), STRIDE)
    return dict(
        workload="N=20 slabs x 40x40 blocks, seed 1000, 64 energies linspace(-3,3), eta=1e-6, 1 k",
        source="oracle/negf_oracle.py solve_point and integrate (tests/golden/make_golden.py)",
        N=int(N), b=int(b), eta=float(eta), energy_index=sel.tolist(), E=E[sel].tolist(),
        transmission=T[sel].tolist(), slab_density=slab[sel].tolist(),
        current=cur[sel].tolist(),
        integrated_slab_density=O.integrate(list(slab), wE).tolist(),
        integrated_current=O.integrate(list(cur), wE).tolist())


if __name__ == "__main__":
    with open(OUT, "w") as f:
        json.dump(compute(), f, indent=1)
        f.write("\n")
    print("wrote", OUT)
