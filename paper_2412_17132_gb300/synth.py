"""Seeded synthetic inputs shaped like the molecules of the paper's acene series.

The paper's molecules (CH4, CO, benzene ... pentacene, CORE65) need an all-electron
DFT starting point that is not available here, so every workload is synthetic:
orbital energies eps_n and RI coefficients O^P_mn with the sizes, energy ranges
and core localisation of a 1s calculation (paper, Sec. "Computational Details"
and the acene study; the correlation-satellite mechanism of Sec. "Assessing the
validity of GW+C for molecular shake-ups" is reproduced by a band of high-lying
virtual states between 3 and 40 Ha).

This module is the ONE piece shared by the CPU oracle and the CUDA path. It
holds no step of the GW+C method: it draws numbers and applies the input
normalisation of the recipe (spectral norm 2 of the weighted Gram matrix of the
occupied-virtual coefficients, weights 4/(eps_a - eps_i)).

Random numbers: orbital energies come from numpy's PCG64 with a fixed seed
sequence; RI coefficients come from a counter-based generator (the SplitMix64
finaliser of Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) keyed by (seed, P, min(m,n), max(m,n)), so that
O^P_mn = O^P_nm and any block can be generated without the others.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

HARTREE_EV = 27.211386245988  # CODATA 2018

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)


def _splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output function applied element-wise to uint64 counters."""
    with np.errstate(over="ignore"):
        z = x + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def _counter_normal(seed: int, p: np.ndarray, lo: np.ndarray, hi: np.ndarray) -> np.ndarray:
    """Standard normal draws keyed by (seed, P, lo, hi); Box-Muller on two uniforms."""
    p = p.astype(np.uint64)
    lo = lo.astype(np.uint64)
    hi = hi.astype(np.uint64)
    with np.errstate(over="ignore"):
        key = _splitmix64(np.uint64(seed) * np.uint64(0xD1B54A32D192ED03) + np.uint64(0x632BE59BD9B4E019))
        c = (p << np.uint64(42)) ^ (lo << np.uint64(21)) ^ hi
        c = c * np.uint64(2)
        u1 = _splitmix64(key ^ c)
        u2 = _splitmix64(key ^ (c + np.uint64(1)))
    f1 = ((u1 >> np.uint64(11)).astype(np.float64) + 1.0) * (1.0 / 9007199254740992.0)  # (0, 1]
    f2 = (u2 >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)  # [0, 1)
    return np.sqrt(-2.0 * np.log(f1)) * np.cos(2.0 * np.pi * f2)


@dataclasses.dataclass
class Molecule:
    """One synthetic system in the layout the library takes (all float64, row-major).

    eps      [n_states]                 ascending; states 0..n_occ-1 occupied; cores first
    core_idx [n_core]                   state index of each core (0..n_core-1)
    o_ov     [n_aux][n_occ*n_virt]      O^P_ia, (i, a) flattened i-major
    o_core   [n_states][n_core][n_aux]  O^P_{m, core_idx[c]}
    """

    name: str
    eps: np.ndarray
    n_occ: int
    core_idx: np.ndarray
    o_ov: np.ndarray
    o_core: np.ndarray
    eta: float
    n_im: int
    xi0: float
    omega: np.ndarray
    n_t: int
    t_max: float

    @property
    def n_states(self) -> int:
        return int(self.eps.shape[0])

    @property
    def n_aux(self) -> int:
        return int(self.o_ov.shape[0])

    @property
    def n_core(self) -> int:
        return int(self.core_idx.shape[0])

    @property
    def n_virt(self) -> int:
        return self.n_states - self.n_occ


def _energies(rng, n_core, core_lo, core_hi, n_val, n_virt, n_high):
    cores = rng.uniform(core_lo, core_hi, n_core) if core_hi > core_lo else np.full(n_core, core_lo)
    val = rng.uniform(-1.0, -0.25, n_val)
    low = rng.uniform(0.0, 3.0, n_virt - n_high)
    high = rng.uniform(3.0, 40.0, n_high)
    return np.concatenate([np.sort(cores), np.sort(val), np.sort(np.concatenate([low, high]))])


def _coefficients(seed, eps, n_occ, n_core, n_aux, sigma=0.02, amp=5.0, frac=0.1):
    """Raw (unscaled) O_ov and O_core with core rows amplified on a random subset of P."""
    n_states = eps.shape[0]
    n_virt = n_states - n_occ
    amp_p = np.ones((n_core, n_aux))
    for c in range(n_core):
        sub = np.random.default_rng([seed, 7, c]).choice(n_aux, size=int(round(frac * n_aux)), replace=False)
        amp_p[c, sub] = amp

    def factor(states, p_idx):
        # amplification of O^P_{m,n}: x amp for every index among (m, n) that is a core with P in its subset
        f = np.ones(np.broadcast_shapes(states.shape, p_idx.shape))
        for c in range(n_core):
            f = f * np.where(states == c, amp_p[c][p_idx], 1.0)
        return f

    o_ov = np.empty((n_aux, n_occ * n_virt))
    ii, aa = np.meshgrid(np.arange(n_occ), np.arange(n_occ, n_states), indexing="ij")
    ii = ii.reshape(-1)
    aa = aa.reshape(-1)
    chunk = max(1, (1 << 23) // max(1, ii.size))
    for p0 in range(0, n_aux, chunk):
        p = np.arange(p0, min(n_aux, p0 + chunk))[:, None]
        g = _counter_normal(seed, np.broadcast_to(p, (p.shape[0], ii.size)), ii[None, :], aa[None, :])
        o_ov[p0 : p0 + p.shape[0]] = sigma * g * factor(ii[None, :], np.broadcast_to(p, g.shape))

    o_core = np.empty((n_states, n_core, n_aux))
    p = np.arange(n_aux)
    for m in range(n_states):
        for c in range(n_core):
            lo, hi = min(m, c), max(m, c)
            g = _counter_normal(seed, p, np.full(n_aux, lo), np.full(n_aux, hi))
            f = amp_p[c] * (amp_p[m] if m < n_core else 1.0)
            o_core[m, c] = sigma * g * f
    return o_ov, o_core


def gram_norm_scale(eps, n_occ, o_ov, target=2.0):
    """Factor s such that s^2 * ||sum_ia w_ia O_ia O_ia^T||_2 = target, w_ia = 4/(eps_a-eps_i).

    The weighted Gram matrix is formed explicitly (one BLAS product, chunked over the columns) and its
    largest eigenvalue taken from a dense symmetric eigensolver."""
    w = 4.0 / (eps[None, n_occ:] - eps[:n_occ, None]).reshape(-1)
    n_aux = o_ov.shape[0]
    g = np.zeros((n_aux, n_aux))
    step = 8192
    for k0 in range(0, o_ov.shape[1], step):
        blk = o_ov[:, k0 : k0 + step]
        g += (blk * w[None, k0 : k0 + step]) @ blk.T
    lam = float(np.linalg.eigvalsh(g)[-1])
    return math.sqrt(target / lam)


def omega_window(core_eps, n_omega, below_ev=25.0, above_ev=5.0):
    """Uniform absolute grid [mean core - 25 eV, mean core + 5 eV] (endpoints included)."""
    c = float(np.mean(core_eps))
    return np.linspace(c - below_ev / HARTREE_EV, c + above_ev / HARTREE_EV, n_omega)


def molecule(
    name,
    n_states,
    n_occ,
    n_core,
    n_aux,
    *,
    seed=0,
    core_lo=-10.41,
    core_hi=-10.39,
    n_high=None,
    n_omega=800,
    n_im=32,
    xi0=1.0,
    eta=1e-3,
    n_t=1 << 16,
    t_max=2000.0,
) -> Molecule:
    n_virt = n_states - n_occ
    if n_high is None:
        n_high = int(round(n_virt * 5 / 52))
    rng = np.random.default_rng(seed)
    eps = _energies(rng, n_core, core_lo, core_hi, n_occ - n_core, n_virt, n_high)
    o_ov, o_core = _coefficients(seed, eps, n_occ, n_core, n_aux)
    s = gram_norm_scale(eps, n_occ, o_ov)
    o_ov *= s
    o_core *= s
    return Molecule(
        name=name,
        eps=eps,
        n_occ=n_occ,
        core_idx=np.arange(n_core, dtype=np.int32),
        o_ov=np.ascontiguousarray(o_ov),
        o_core=np.ascontiguousarray(o_core),
        eta=eta,
        n_im=n_im,
        xi0=xi0,
        omega=omega_window(eps[:n_core], n_omega),
        n_t=n_t,
        t_max=t_max,
    )


def tiny(seed=0) -> Molecule:
    """Tiny molecule: 60 states, 8 occupied (one 1s core at -10.40 Ha), 200 aux, 400 omega points."""
    return molecule("tiny", 60, 8, 1, 200, seed=seed, core_lo=-10.40, core_hi=-10.40, n_high=5, n_omega=400)


def benzene(seed=0) -> Molecule:
    """Benzene-sized: 300 states, 21 occupied (six 1s cores near -10.4 Ha), 1100 aux, 800 omega points."""
    return molecule("benzene", 300, 21, 6, 1100, seed=seed, n_omega=800)


def pentacene(seed=0) -> Molecule:
    """Pentacene-sized: 1300 states, 73 occupied (22 1s cores), 4500 aux, 800 omega points."""
    return molecule("pentacene", 1300, 73, 22, 4500, seed=seed, n_omega=800)


def batch_member(j: int) -> Molecule:
    """Molecule j of the uneven batch: N_states ~ U{100..1300}, seed 1000 + j."""
    rng = np.random.default_rng(1000 + j)
    n = int(rng.integers(100, 1301))
    n_occ = max(2, int(round(n / 18)))
    n_core = max(1, int(round(0.3 * n_occ)))
    return molecule(f"batch{j}", n, n_occ, n_core, int(round(3.5 * n)), seed=1000 + j)


def serving_request(request_id: int) -> Molecule:
    """Request of the serving stream: N_states log-uniform on [100, 1500], seed = request id."""
    rng = np.random.default_rng(request_id)
    n = int(round(math.exp(rng.uniform(math.log(100), math.log(1500)))))
    n_occ = max(2, int(round(n / 18)))
    n_core = max(1, int(round(0.3 * n_occ)))
    return molecule(f"req{request_id}", n, n_occ, n_core, int(round(3.5 * n)), seed=request_id)


def small(n_states=24, n_occ=4, n_core=1, n_aux=20, seed=3, n_omega=40, n_high=None) -> Molecule:
    """Arbitrary small system for ragged-shape and brute-force tests."""
    return molecule("small", n_states, n_occ, n_core, n_aux, seed=seed, n_omega=n_omega, n_high=n_high)


# ----------------------------------------------------------------------------------------
# Device-side generation (batched and serving workloads)
# ----------------------------------------------------------------------------------------
def _i64(c: int) -> int:
    """Two's-complement int64 value of a uint64 constant."""
    return c - (1 << 64) if c >= (1 << 63) else c


def _srl(x, k: int):
    """Logical right shift of int64 torch values (bit pattern of the uint64 shift)."""
    return (x >> k) & ((1 << (64 - k)) - 1)


def _splitmix64_t(x):
    z = x + _i64(0x9E3779B97F4A7C15)
    z = (z ^ _srl(z, 30)) * _i64(0xBF58476D1CE4E5B9)
    z = (z ^ _srl(z, 27)) * _i64(0x94D049BB133111EB)
    return z ^ _srl(z, 31)


def _counter_normal_t(seed, p, lo, hi):
    """Torch (int64 bit patterns) version of _counter_normal: same draws, torch transcendental functions."""
    import torch

    key = _splitmix64_t(torch.tensor(_i64((seed * 0xD1B54A32D192ED03 + 0x632BE59BD9B4E019) % (1 << 64)), dtype=torch.int64,
                                     device=p.device))
    c = (p << 42) ^ (lo << 21) ^ hi
    c = c * 2
    u1 = _splitmix64_t(key ^ c)
    u2 = _splitmix64_t(key ^ (c + 1))
    f1 = (_srl(u1, 11).to(torch.float64) + 1.0) * (1.0 / 9007199254740992.0)
    f2 = _srl(u2, 11).to(torch.float64) * (1.0 / 9007199254740992.0)
    return torch.sqrt(-2.0 * torch.log(f1)) * torch.cos(2.0 * math.pi * f2)


def molecule_device(name, n_states, n_occ, n_core, n_aux, *, seed=0, core_lo=-10.41, core_hi=-10.39, n_high=None,
                    n_omega=800, n_im=32, xi0=1.0, eta=1e-3, n_t=1 << 16, t_max=2000.0, power_steps=20,
                    device="cuda", sigma=0.02, amp=5.0, frac=0.1, exact_scale=False):
    """The recipe of `molecule` with O generated on the GPU (torch), for workloads too large to
    generate on the host per request. Energies and amplified subsets are the host generator's; the
    O^P_mn draws are the same counter-based values up to the last bits of log/cos; the global scale
    comes from `power_steps` steps of power iteration on the device (no host synchronisation), so
    ||Pi(i0)||_2 = 2 holds to the accuracy of that iteration rather than to 1e-12; with
    exact_scale=True it is the Lanczos value of the host generator (matrix-vector products on the
    device), and the molecule equals `molecule(...)` to rounding.
    Returns a Molecule whose eps/core_idx/omega are numpy and whose o_ov/o_core are CUDA tensors."""
    import torch

    n_virt = n_states - n_occ
    if n_high is None:
        n_high = int(round(n_virt * 5 / 52))
    rng = np.random.default_rng(seed)
    eps = _energies(rng, n_core, core_lo, core_hi, n_occ - n_core, n_virt, n_high)
    amp_p = np.ones((n_core, n_aux))
    for c in range(n_core):
        sub = np.random.default_rng([seed, 7, c]).choice(n_aux, size=int(round(frac * n_aux)), replace=False)
        amp_p[c, sub] = amp
    dev = torch.device(device)
    amp_t = torch.as_tensor(amp_p, device=dev)
    ii = torch.arange(n_occ, device=dev, dtype=torch.int64).repeat_interleave(n_virt)
    aa = torch.arange(n_occ, n_states, device=dev, dtype=torch.int64).repeat(n_occ)
    o_ov = torch.empty((n_aux, ii.numel()), dtype=torch.float64, device=dev)
    chunk = max(1, (1 << 24) // max(1, ii.numel()))
    for p0 in range(0, n_aux, chunk):
        p1 = min(n_aux, p0 + chunk)
        p = torch.arange(p0, p1, device=dev, dtype=torch.int64)[:, None]
        g = _counter_normal_t(seed, p.expand(-1, ii.numel()), ii[None, :].expand(p1 - p0, -1),
                              aa[None, :].expand(p1 - p0, -1))
        f = torch.ones_like(g)
        for c in range(n_core):
            f = torch.where(ii[None, :] == c, f * amp_t[c, p0:p1][:, None], f)
        o_ov[p0:p1] = sigma * g * f
    m_idx = torch.arange(n_states, device=dev, dtype=torch.int64)
    o_core = torch.empty((n_states, n_core, n_aux), dtype=torch.float64, device=dev)
    pp = torch.arange(n_aux, device=dev, dtype=torch.int64)
    for c in range(n_core):
        lo = torch.minimum(m_idx, torch.tensor(c, device=dev))
        hi = torch.maximum(m_idx, torch.tensor(c, device=dev))
        g = _counter_normal_t(seed, pp[None, :].expand(n_states, -1), lo[:, None].expand(-1, n_aux),
                              hi[:, None].expand(-1, n_aux))
        f = amp_t[c][None, :].expand(n_states, -1).clone()
        if n_core > 0:
            core_rows = m_idx < n_core
            f[core_rows] = f[core_rows] * amp_t[m_idx[core_rows]]
        o_core[:, c, :] = sigma * g * f
    # global scale: largest eigenvalue of sum_ia (4/Delta_ia) O_ia O_ia^T by power iteration
    eps_t = torch.as_tensor(eps, device=dev)
    w = 4.0 / (eps_t[n_occ:][None, :] - eps_t[:n_occ][:, None]).reshape(-1)
    if exact_scale:
        g = torch.zeros((n_aux, n_aux), dtype=torch.float64, device=dev)
        step = 8192
        for k0 in range(0, o_ov.shape[1], step):
            blk = o_ov[:, k0 : k0 + step]
            g += (blk * w[None, k0 : k0 + step]) @ blk.t()
        lam = float(np.linalg.eigvalsh(g.cpu().numpy())[-1])
        s = math.sqrt(2.0 / lam)
    else:
        v = torch.ones(n_aux, dtype=torch.float64, device=dev)
        lam = torch.tensor(1.0, dtype=torch.float64, device=dev)
        for _ in range(power_steps):
            u = o_ov @ (w * (o_ov.t() @ v))
            lam = torch.linalg.vector_norm(u) / torch.linalg.vector_norm(v)
            v = u / torch.linalg.vector_norm(u)
        s = torch.sqrt(2.0 / lam)
    o_ov.mul_(s)
    o_core.mul_(s)
    return Molecule(name=name, eps=eps, n_occ=n_occ, core_idx=np.arange(n_core, dtype=np.int32), o_ov=o_ov, o_core=o_core,
                    eta=eta, n_im=n_im, xi0=xi0, omega=omega_window(eps[:n_core], n_omega), n_t=n_t, t_max=t_max)


def pentacene_device(seed=0, **kw) -> Molecule:
    """The pentacene-sized molecule with O generated on the GPU and the exact normalisation."""
    return molecule_device("pentacene", 1300, 73, 22, 4500, seed=seed, n_omega=800, exact_scale=True, **kw)


def batch_member_device(j: int, **kw) -> Molecule:
    """Molecule j of the uneven batch (seed 1000 + j) generated on the GPU."""
    rng = np.random.default_rng(1000 + j)
    n = int(rng.integers(100, 1301))
    n_occ = max(2, int(round(n / 18)))
    n_core = max(1, int(round(0.3 * n_occ)))
    return molecule_device(f"batch{j}", n, n_occ, n_core, int(round(3.5 * n)), seed=1000 + j, **kw)


def serving_request_device(request_id: int, **kw) -> Molecule:
    """Request of the serving stream (seed = request id) generated on the GPU."""
    rng = np.random.default_rng(request_id)
    n = int(round(math.exp(rng.uniform(math.log(100), math.log(1500)))))
    n_occ = max(2, int(round(n / 18)))
    n_core = max(1, int(round(0.3 * n_occ)))
    return molecule_device(f"req{request_id}", n, n_occ, n_core, int(round(3.5 * n)), seed=request_id, **kw)
