"""Pins of the oracle's atom-block scattering self-energies (Sigma block-diagonal with one A x A
block per atom) against dense inversion of Eqs. (1)-(2), the orbital-diagonal form it reduces to
at A = 1, and current conservation of the elastic Born iteration of Eq. (4)."""
import numpy as np
import pytest

import oracle as O
from workloads import make_device, channel_device

KT = O.KT_300K


def _block_scatter(N, b, A, seed, gamma=0.05, f=0.7):
    """Physical atom-block self-energies: Sigma^R = R - i G, Sigma^< = 2 i f G with G Hermitian
    positive semi-definite and R Hermitian per A x A block."""
    rng = np.random.default_rng(seed)
    sR = np.zeros((N, b, b), dtype=complex)
    sL = np.zeros_like(sR)
    for i in range(N):
        for a in range(b // A):
            X = rng.normal(size=(A, A)) + 1j * rng.normal(size=(A, A))
            G = gamma * (X @ X.conj().T) / A
            Y = 0.02 * (rng.normal(size=(A, A)) + 1j * rng.normal(size=(A, A)))
            R = 0.5 * (Y + Y.conj().T)
            sl = slice(a * A, (a + 1) * A)
            sR[i, sl, sl] = R - 1j * G
            sL[i, sl, sl] = 2j * f * G
    return sR, sL


def test_atom_block_layout_round_trip_and_a1_is_the_diagonal():
    rng = np.random.default_rng(1)
    b, A = 6, 3
    X = rng.normal(size=(b, b)) + 1j * rng.normal(size=(b, b))
    row = O.atom_blocks(X, A)
    assert row.shape == (b * A,)
    # entry (r, c) of a block at r A + c mod A
    assert row[4 * A + (5 % A)] == X[4, 5] and row[1 * A + (0 % A)] == X[1, 0]
    B = O.atom_block_matrix(row, b, A)
    for r in range(b):
        for c in range(b):
            assert B[r, c] == (X[r, c] if r // A == c // A else 0)
    assert np.array_equal(O.atom_blocks(X, 1), np.diag(X))
    assert np.array_equal(O.atom_block_matrix(np.diag(X), b, 1), np.diag(np.diag(X)))


@pytest.mark.parametrize("N,b,A", [(1, 4, 2), (3, 4, 2), (4, 6, 3), (3, 5, 5)])
def test_rgf_with_atom_blocks_equals_dense_inverse(N, b, A):
    dev = make_device(N, b, 31 + N * b + A)
    V = np.random.default_rng(7).uniform(-0.3, 0.3, (N, b))
    E, eta = -0.21, 1e-6
    leads = O.lead_self_energies(dev.D, dev.T, E, eta, 0.1, -0.1, KT)
    sR, sL = _block_scatter(N, b, A, 5)
    r = O.rgf(dev.D, dev.T, E, eta, V, leads, sR, sL)
    G, GL = O.dense_green(dev.D, dev.T, E, eta, V, leads, sR, sL)
    scale = max(np.abs(G).max(), 1.0)
    scale_l = max(np.abs(GL).max(), 1e-300)
    for i in range(N):
        s = slice(i * b, (i + 1) * b)
        assert np.abs(r["G"][i] - G[s, s]).max() < 1e-11 * scale
        assert np.abs(r["GL"][i] - GL[s, s]).max() < 1e-11 * scale_l
    for i in range(N - 1):
        s, t = slice((i + 1) * b, (i + 2) * b), slice(i * b, (i + 1) * b)
        assert np.abs(r["GLoff"][i] - GL[s, t]).max() < 1e-11 * scale_l


def test_diagonal_atom_blocks_give_the_orbital_diagonal_solution():
    """Atom blocks that happen to be diagonal are the orbital-diagonal form."""
    N, b, A = 3, 4, 2
    dev = make_device(N, b, 77)
    rng = np.random.default_rng(2)
    g = 0.05 * rng.random((N, b))
    dR, dL = 0.01 * rng.normal(size=(N, b)) - 1j * g, 1.4j * g
    mR = np.array([np.diag(x) for x in dR])
    mL = np.array([np.diag(x) for x in dL])
    a = O.solve_point(dev.D, dev.T, 0.3, 1e-6, sR=dR, sL=dL)
    c = O.solve_point(dev.D, dev.T, 0.3, 1e-6, sR=mR, sL=mL)
    for key in ("density", "current", "diagGR", "diagGL"):
        assert np.allclose(a[key], c[key], rtol=0, atol=1e-13 * max(np.abs(a[key]).max(), 1e-30))


def test_acoustic_born_iteration_with_atom_blocks_conserves_current():
    """Elastic scattering with Sigma^{R,<} = D_ac (atom blocks of G^{R,<}) conserves the bond
    current at every energy at convergence (Tr over a block of Sigma^< G^> - Sigma^> G^< is
    zero entry by entry); a wrong block layout (mixing atoms) breaks it."""
    N, b, A = 5, 4, 2
    dev = channel_device(N, b, 23)
    E = np.linspace(-0.2, 0.2, 5)
    assert all(np.all(np.abs(e - dev.meta["d"]) < 2 * dev.meta["t"]) for e in E)

    def run(layout_ok):
        sR = np.zeros((len(E), N * b * A), dtype=complex)
        sL = np.zeros_like(sR)
        for _ in range(300):
            outs = []
            for i, e in enumerate(E):
                mR = np.array([O.atom_block_matrix(x, b, A) for x in sR[i].reshape(N, b * A)])
                mL = np.array([O.atom_block_matrix(x, b, A) for x in sL[i].reshape(N, b * A)])
                if not layout_ok:  # couple atom 0 of each slab to itself transposed
                    mR = np.transpose(mR, (0, 2, 1))
                outs.append(O.solve_point(dev.D, dev.T, e, 0.0, None, eta_lead=1e-7, sR=mR,
                                          sL=mL))
            dGR = np.array([np.concatenate([O.atom_blocks(x, A) for x in o["blocks"]["G"]])
                            for o in outs])[None]
            dGL = np.array([np.concatenate([O.atom_blocks(x, A) for x in o["blocks"]["GL"]])
                            for o in outs])[None]
            sR, sL, delta = O.scba_step(dGR, dGL, np.ones(1), 0.05, 0.0, 3, 0.1, sR, sL)
            if delta < 1e-14:
                break
        worst = 0.0
        for o in outs:
            j = o["current"]
            worst = max(worst, np.abs(j - j.mean()).max() / max(np.abs(j).max(), 1e-12))
        return delta, worst

    delta, worst = run(True)
    assert delta < 1e-12 and worst < 1e-9
    _, worst_bad = run(False)
    assert worst_bad > 1e-6
