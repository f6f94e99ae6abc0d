"""Interface couplings (hoppings nonzero only between the facing atoms of neighbouring slabs):
the sweeps restricted to the r x c support give the dense sweeps' results and the oracle's."""
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


def _t(x):
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


def _solve(dev, E, opt, iface, V=None):
    d = negf.Device(_t(dev.D[None]), _t(dev.T[None]), iface=iface)
    Et = _t(E)
    st = torch.zeros(len(E), dtype=torch.int32, device="cuda")
    lead = negf.lead_selfenergy(d, Et, st, opt)
    out = negf.rgf_solve(d, Et, st, lead["sigma_R"], lead["sigma_L"], opt,
                         V=None if V is None else _t(V))
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items() if isinstance(v, torch.Tensor)}


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("N,b,r,c", [(6, 60, 20, 30), (4, 140, 40, 40), (3, 50, 50, 10)])
def test_interface_sweeps_match_dense_and_oracle(prec, N, b, r, c):
    dev = make_device(N, b, 900 + b + r, ge_frac=0.1, iface=(r, c))
    E = np.linspace(-1.6, 1.3, 6)
    V = np.random.default_rng(b).uniform(-0.1, 0.1, (N, b))
    opt = negf.options(precision=prec)
    sparse = _solve(dev, E, opt, (r, c), V)
    dense = _solve(dev, E, opt, None, V)
    refs = [O.solve_point(dev.D, dev.T, e, 1e-6, V) for e in E]
    tol = 1e-9 if prec == 0 else 1e-6
    scale = max(np.abs(x["density"]).max() for x in refs)
    jscale = max(np.abs(x["current"]).max() for x in refs)
    for p, x in enumerate(refs):
        for out in (sparse, dense):
            assert np.abs(out["density"][p] - x["density"]).max() <= tol * scale
            assert np.abs(out["current"][p] - x["current"]).max() <= tol * jscale
            assert abs(out["transmission"][p] - x["transmission"]) <= \
                tol * max(1.0, abs(x["transmission"]))
    assert np.all(sparse["status"] == 0)
    if prec == 0:
        # the same nonzero terms, summed in another order (the GEMMs contract over r or c
        # instead of b); the decimation amplifies that rounding difference near its
        # ill-conditioned steps (cond(z - eps_n) ~ 1e7 at band edges), hence 1e-10, not 1e-15
        assert np.abs(sparse["density"] - dense["density"]).max() <= 1e-10 * scale


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("N,b,r,c", [(5, 60, 20, 30), (3, 96, 8, 40), (4, 50, 50, 10)])
def test_interface_decimation_matches_dense_and_oracle(prec, N, b, r, c):
    """The decimation restricted to the support of alpha_n, beta_n gives the dense decimation's
    self-energies; Sigma_L lives on the first c rows / columns, Sigma_R on the last r."""
    dev = make_device(N, b, 1700 + b + r, ge_frac=0.1, iface=(r, c))
    E = np.concatenate([np.linspace(-1.7, 1.4, 5), [-0.499]])
    opt = negf.options(precision=prec)
    Et = _t(E)
    st = torch.zeros(len(E), dtype=torch.int32, device="cuda")
    out = {}
    for key, iface in (("sparse", (r, c)), ("dense", None)):
        d = negf.Device(_t(dev.D[None]), _t(dev.T[None]), iface=iface)
        lead = negf.lead_selfenergy(d, Et, st, opt)
        torch.cuda.synchronize()
        out[key] = {k: v.cpu().numpy() for k, v in lead.items()}
    sp, dn = out["sparse"], out["dense"]
    assert np.all(sp["status"] == 0) and np.all(dn["status"] == 0)
    o = negf.options()
    tol = 1e-9 if prec == 0 else 1e-6
    for p, e in enumerate(E):
        x = O.lead_self_energies(dev.D, dev.T, e, o.eta_lead, o.mu_L, o.mu_R, o.kT)
        for side, ref in ((0, x["sigL"]), (1, x["sigR"])):
            sc = max(np.abs(ref).max(), 1e-300)
            for res in (sp, dn):
                assert np.abs(res["sigma_R"][p, side] - ref).max() <= tol * sc, (p, side)
        sl, sr = sp["sigma_R"][p, 0], sp["sigma_R"][p, 1]
        assert np.all(sl[c:, :] == 0) and np.all(sl[:, c:] == 0)
        assert np.all(sr[:b - r, :] == 0) and np.all(sr[:, :b - r] == 0)
    if prec == 0:
        sc = np.abs(dn["sigma_R"]).max()
        assert np.abs(sp["sigma_R"] - dn["sigma_R"]).max() <= 1e-10 * sc
        assert np.abs(sp["iters"] - dn["iters"]).max() <= 1


@pytest.mark.parametrize("prec,seg", [(0, 0), (0, 2), (1, 0)])
@pytest.mark.parametrize("N,b,r,c", [(5, 40, 10, 20), (4, 60, 60, 15), (3, 30, 7, 30)])
def test_interface_adjoint_matches_dense_and_oracle(prec, seg, N, b, r, c):
    """dL/dV with the adjoint's products restricted to the hopping support equals the dense
    adjoint and the oracle's dense gradient, with and without sweep checkpointing."""
    dev = make_device(N, b, 2100 + b + r, ge_frac=0.1, iface=(r, c))
    rng = np.random.default_rng(b + c)
    E = np.array([-0.9, 0.15, 1.1])
    V = rng.uniform(-0.2, 0.2, (N, b))
    cb = rng.normal(size=(len(E), N * b))
    db = rng.normal(size=(len(E), N - 1))
    opt = negf.options(precision=prec, adjoint_segment=seg)
    Et = _t(E)
    st = torch.zeros(len(E), dtype=torch.int32, device="cuda")
    grads = {}
    for key, iface in (("sparse", (r, c)), ("dense", None)):
        d = negf.Device(_t(dev.D[None]), _t(dev.T[None]), iface=iface)
        lead = negf.lead_selfenergy(d, Et, st, opt)
        Vbar, status = negf.rgf_adjoint(d, Et, st, lead["sigma_R"], lead["sigma_L"], opt,
                                        density_bar=_t(cb), current_bar=_t(db), V=_t(V))
        torch.cuda.synchronize()
        assert np.all(status.cpu().numpy() == 0)
        grads[key] = Vbar.cpu().numpy()
    ref = np.zeros((N, b))
    for p, e in enumerate(E):
        leads = O.lead_self_energies(dev.D, dev.T, e, 1e-6, 0.1, -0.1, O.KT_300K)
        ref += O.gradient_dense(dev.D, dev.T, e, 1e-6, V, leads, cb[p], db[p])
    tol = 1e-7 if prec == 0 else 1e-6
    scale = np.abs(ref).max()
    for g in grads.values():
        assert np.abs(g - ref).max() <= tol * scale
    if prec == 0:  # same nonzero terms, summed in another order
        assert np.abs(grads["sparse"] - grads["dense"]).max() <= 1e-10 * scale


def test_interface_adjoint_from_solve_checkpoints():
    N, b, r, c = 5, 40, 10, 20
    dev = make_device(N, b, 2222, ge_frac=0.1, iface=(r, c))
    rng = np.random.default_rng(3)
    E = np.array([-0.9, 0.15, 1.1])
    V = _t(rng.uniform(-0.2, 0.2, (N, b)))
    cb, db = _t(rng.normal(size=(len(E), N * b))), _t(rng.normal(size=(len(E), N - 1)))
    opt = negf.options(precision=1)
    d = negf.Device(_t(dev.D[None]), _t(dev.T[None]), iface=(r, c))
    Et = _t(E)
    st = torch.zeros(len(E), dtype=torch.int32, device="cuda")
    lead = negf.lead_selfenergy(d, Et, st, opt)
    g0, _ = negf.rgf_adjoint(d, Et, st, lead["sigma_R"], lead["sigma_L"], opt, density_bar=cb,
                             current_bar=db, V=V)
    ck = negf.checkpoint_buffer(d, len(E))
    negf.rgf_solve(d, Et, st, lead["sigma_R"], lead["sigma_L"], opt, V=V, checkpoints=ck)
    g1, st1 = negf.rgf_adjoint(d, Et, st, lead["sigma_R"], lead["sigma_L"], opt, density_bar=cb,
                               current_bar=db, V=V, checkpoints=ck)
    torch.cuda.synchronize()
    assert np.all(st1.cpu().numpy() == 0)
    g0, g1 = g0.cpu().numpy(), g1.cpu().numpy()
    assert np.abs(g1 - g0).max() <= 1e-12 * np.abs(g0).max()
