"""Seeded synthetic device Hamiltonians and grids.

The paper's devices (Sec. "Overview of the problem": ~24,000 atoms, sp3d5s* tight binding with
10 orbitals per atom, Si with 10% Ge) cannot be rebuilt without tight-binding parameter tables,
so these generators stand in for them with the same shapes:

* a block-tridiagonal Hamiltonian of N slabs, each slab holding ``b = 10 * atoms`` orbitals;
* on-site blocks D_i Hermitian with diagonal U(lo, hi) eV and complex off-diagonal entries of
  standard deviation ``sigma_on * sqrt(40 / b)`` (so b = 40 gives N(0, 0.3));
* hopping blocks H_{i,i+1} with complex entries of standard deviation ``1 / sqrt(b)``;
* an optional transverse-k dependence H_ii(k) = D_i + W_i e^{ik} + W_i^H e^{-ik} with W_i complex
  of standard deviation ``w_scale / sqrt(b)`` (k-independent hoppings);
* a random alloy: every atom is Ge with probability ``ge_frac`` and then shifts the diagonal of
  its 10 orbitals by ``ge_shift`` eV.

Every array is complex128 row-major; ``Hu[i]`` is the coupling H_{i,i+1} between slab i and
slab i+1 (0-based), and H_{i+1,i} = Hu[i]^H.  Seeds follow ``1000 * config + sample``.
Nothing here computes a Green's function.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

ORBITALS_PER_ATOM = 10


@dataclass
class Device:
    """Block-tridiagonal device: on-site blocks D, k-dependent part W, hoppings T."""

    N: int
    b: int
    D: np.ndarray                     # [N, b, b] complex128, Hermitian
    T: np.ndarray                     # [N-1, b, b] complex128, T[i] = H_{i,i+1}
    W: Optional[np.ndarray] = None    # [N, b, b] complex128 or None
    ge_mask: Optional[np.ndarray] = None  # [N, b // 10] bool
    meta: dict = field(default_factory=dict)


def _complex_normal(rng, shape, std):
    s = std / np.sqrt(2.0)
    return rng.normal(0.0, s, shape) + 1j * rng.normal(0.0, s, shape)


def make_device(N: int, b: int, seed: int, *, sigma_on: float = 0.3, diag_lo: float = -2.0,
                diag_hi: float = 2.0, ge_frac: float = 0.0, ge_shift: float = 0.2,
                with_k: bool = False, w_scale: float = 0.1,
                hop_std: Optional[float] = None, iface: Optional[tuple] = None) -> Device:
    """Draw one seeded device (all blocks complex128).

    iface=(r, c): interface couplings -- every hopping block H_{i,i+1} keeps only its last r
    rows and first c columns (the orbitals of the atoms facing the neighbouring slab), the rest
    is zero; the random draws are the same as without it."""
    if N < 1 or b < 1:
        raise ValueError("N and b must be positive")
    rng = np.random.default_rng(seed)
    std_on = sigma_on * np.sqrt(40.0 / b)
    hop = (1.0 / np.sqrt(b)) if hop_std is None else hop_std
    D = np.empty((N, b, b), dtype=np.complex128)
    iu = np.triu_indices(b, 1)
    for i in range(N):
        blk = np.zeros((b, b), dtype=np.complex128)
        blk[iu] = _complex_normal(rng, iu[0].size, std_on)
        blk = blk + blk.conj().T
        blk[np.diag_indices(b)] = rng.uniform(diag_lo, diag_hi, b)
        D[i] = blk
    ge_mask = None
    if ge_frac > 0.0:
        n_atoms = max(1, b // ORBITALS_PER_ATOM)
        ge_mask = rng.random((N, n_atoms)) < ge_frac
        for i in range(N):
            for a in np.nonzero(ge_mask[i])[0]:
                lo = a * ORBITALS_PER_ATOM
                hi = min(b, lo + ORBITALS_PER_ATOM)
                idx = np.arange(lo, hi)
                D[i, idx, idx] += ge_shift
    T = _complex_normal(rng, (max(N - 1, 0), b, b), hop)
    W = _complex_normal(rng, (N, b, b), w_scale / np.sqrt(b)) if with_k else None
    if iface is not None:
        r, c = iface
        mask = np.zeros((b, b), dtype=bool)
        mask[b - r:, :c] = True
        T = np.where(mask[None], T, 0.0)
    return Device(N=N, b=b, D=D, T=T, W=W, ge_mask=ge_mask,
                  meta=dict(seed=seed, sigma_on=sigma_on, ge_frac=ge_frac, with_k=with_k,
                            iface=iface))


def hamiltonian_k(dev: Device, k: float):
    """Blocks of H(k): returns (Hd [N,b,b], Hu [N-1,b,b]) as complex128 copies."""
    if dev.W is None:
        return dev.D.copy(), dev.T.copy()
    ph = np.exp(1j * k)
    Hd = dev.D + dev.W * ph + np.conj(np.swapaxes(dev.W, 1, 2)) * np.conj(ph)
    return Hd, dev.T.copy()


def chain_device(N: int, eps: float = 0.0, t: float = 1.0) -> Device:
    """1D nearest-neighbour chain (b = 1): on-site eps, hopping t."""
    D = np.full((N, 1, 1), eps, dtype=np.complex128)
    T = np.full((max(N - 1, 0), 1, 1), t, dtype=np.complex128)
    return Device(N=N, b=1, D=D, T=T, meta=dict(kind="chain", eps=eps, t=t))


def channel_device(N: int, b: int, seed: int, *, d_lo: float = -1.0, d_hi: float = 1.0,
                   t_lo: float = 0.5, t_hi: float = 1.5) -> Device:
    """b decoupled chains hidden behind one random unitary U shared by every slab.

    H_ii = U diag(d) U^H and H_{i,i+1} = U diag(t) U^H, so channel c is a clean chain with
    on-site d_c and hopping t_c; the blocks themselves are dense and complex.
    Returns the device with ``meta['d']`` and ``meta['t']`` holding the channel parameters.
    """
    rng = np.random.default_rng(seed)
    Z = _complex_normal(rng, (b, b), 1.0)
    U, _ = np.linalg.qr(Z)
    d = rng.uniform(d_lo, d_hi, b)
    tc = rng.uniform(t_lo, t_hi, b)
    on = (U * d) @ U.conj().T
    on = 0.5 * (on + on.conj().T)
    hop = (U * tc) @ U.conj().T
    D = np.broadcast_to(on, (N, b, b)).copy()
    T = np.broadcast_to(hop, (max(N - 1, 0), b, b)).copy()
    return Device(N=N, b=b, D=D, T=T, meta=dict(kind="channels", d=d, t=tc))


def energy_grid_linspace(lo: float, hi: float, n: int):
    """Uniform grid with trapezoid weights."""
    E = np.linspace(lo, hi, n)
    w = np.full(n, (hi - lo) / (n - 1) if n > 1 else 1.0)
    if n > 1:
        w[0] *= 0.5
        w[-1] *= 0.5
    return E, w


def energy_grid_uniform(e0: float, dE: float, n: int):
    """E_j = e0 + j dE with rectangle weights dE (the homogeneous SCBA mesh)."""
    E = e0 + dE * np.arange(n)
    return E, np.full(n, dE)


def k_grid(n_k: int):
    """k_m = -pi + 2 pi (m + 1/2) / n_k with weights 1/n_k; a single point is k = 0."""
    if n_k == 1:
        return np.zeros(1), np.ones(1)
    k = -np.pi + 2.0 * np.pi * (np.arange(n_k) + 0.5) / n_k
    return k, np.full(n_k, 1.0 / n_k)


def random_potential(N: int, b: int, seed: int, amp: float = 0.3, per_atom: bool = True):
    """On-site potential per orbital [N, b]; per_atom draws one U(-amp, amp) value per atom."""
    rng = np.random.default_rng(seed)
    if per_atom:
        n_atoms = -(-b // ORBITALS_PER_ATOM)
        va = rng.uniform(-amp, amp, (N, n_atoms))
        return np.repeat(va, ORBITALS_PER_ATOM, axis=1)[:, :b].copy()
    return rng.uniform(-amp, amp, (N, b))


# The five workloads the throughput and parity targets are stated on.
CONFIGS = {
    0: dict(name="ballistic_N20_b40", N=20, b=40, n_E=64, E_lo=-3.0, E_hi=3.0, n_k=1,
            ge_frac=0.0, eta=1e-6),
    1: dict(name="ballistic_N70_b400_alloy", N=70, b=400, n_E=512, E_lo=-3.0, E_hi=3.0,
            n_k=8, ge_frac=0.1, eta=1e-6),
    2: dict(name="batched_ragged_b200-800", N=70, b_choices=(200, 300, 400, 500, 600, 700, 800),
            n_samples=128, n_E=256, E_lo=-3.0, E_hi=3.0, n_k=4, ge_frac=0.1, eta=1e-6),
    3: dict(name="scba_N70_b600", N=70, b=600, n_E=1024, E0=-2.56, dE=0.005, n_k=1,
            ge_frac=0.0, eta=1e-6, D_ac=0.01, D_op=0.01, hw=0.060, kT=0.025852, n_iter=20),
    4: dict(name="adjoint_N70_b3430", N=70, b=3430, n_E=1024, E_lo=-3.0, E_hi=3.0, n_k=1,
            ge_frac=0.0, eta=1e-6, V_amp=0.3),
}


def config_workload(cfg: int, sample: int = 0, *, N: Optional[int] = None,
                    b: Optional[int] = None, n_E: Optional[int] = None,
                    n_k: Optional[int] = None):
    """Device + grids of one configuration; N, b, n_E, n_k may be reduced for small copies."""
    c = dict(CONFIGS[cfg])
    seed = 1000 * cfg + sample
    if cfg == 2 and b is None:
        b = int(np.random.default_rng(seed).choice(c["b_choices"]))
    N = c["N"] if N is None else N
    b = c["b"] if b is None else b
    n_E = c["n_E"] if n_E is None else n_E
    n_k = c["n_k"] if n_k is None else n_k
    dev = make_device(N, b, seed, ge_frac=c.get("ge_frac", 0.0), with_k=n_k > 1)
    if "dE" in c:
        E, wE = energy_grid_uniform(c["E0"], c["dE"], n_E)
    else:
        E, wE = energy_grid_linspace(c["E_lo"], c["E_hi"], n_E)
    k, wk = k_grid(n_k)
    out = dict(cfg=cfg, name=c["name"], device=dev, E=E, wE=wE, k=k, wk=wk, eta=c["eta"],
               seed=seed, params=c)
    if cfg == 4:
        out["V"] = random_potential(N, b, seed + 500, c["V_amp"])
    return out
