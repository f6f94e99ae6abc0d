"""Adaptive non-uniform energy meshes (host logic, CPU): a narrow Lorentzian resonance, whose
integral is known in closed form, is integrated to the requested accuracy with points gathered
around the resonance and far fewer than a uniform mesh of the same accuracy needs."""
import numpy as np

from paper_1510_04686_gb300.mesh import refine_mesh, trapezoid_weights


def _lorentz(E0, g):
    return lambda E: np.stack([g / ((np.asarray(E) - E0) ** 2 + g ** 2),
                               0.5 * np.ones(len(E))], axis=1)


def test_refine_mesh_integrates_a_narrow_resonance():
    E0, g = 0.137, 1e-3
    exact = np.arctan((1.0 - E0) / g) + np.arctan((1.0 + E0) / g)
    calls = []

    def ev(E):
        calls.append(len(E))
        return _lorentz(E0, g)(E)
    E, F, w, rounds = refine_mesh(ev, -1.0, 1.0, n_init=17, tol=1e-5, max_points=20000)
    assert np.all(np.diff(E) > 0) and len(E) == len(F) == len(w)
    got = (w * F[:, 0]).sum()
    assert abs(got - exact) / exact < 1e-4
    assert abs((w * F[:, 1]).sum() - 1.0) < 1e-13     # a constant is integrated exactly
    near = np.abs(E - E0) < 20 * g
    assert near.sum() > 0.5 * len(E)                   # the points gather at the resonance
    # a uniform trapezoid mesh with this many points (spacing about the resonance width) misses
    # the integral by far more (once the spacing is well below the width the uniform rule
    # converges very fast on a Lorentzian, so the comparison is made at this budget)
    Eu = np.linspace(-1.0, 1.0, len(E))
    err_u = abs((trapezoid_weights(Eu) * _lorentz(E0, g)(Eu)[:, 0]).sum() - exact) / exact
    assert err_u > 10 * abs(got - exact) / exact
    assert sum(calls) == len(E) and len(calls) == rounds + 1


def test_refine_mesh_stops_at_its_budget():
    E, F, w, rounds = refine_mesh(_lorentz(0.0, 1e-6), -1.0, 1.0, n_init=9, tol=1e-12,
                                  max_points=200)
    assert len(E) <= 200 and abs(w.sum() - 2.0) < 1e-14
