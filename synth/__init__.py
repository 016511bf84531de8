"""Seeded synthetic inputs shared by the oracle side and the CUDA side.

This module holds no arithmetic of the method (no bias, no CV, no force, no
integrator): it only places atoms, picks index subsets and draws hill
centres/heights and evaluation points, all from numpy's PCG64 generator with
an explicit seed.  Both the tests and the benchmark build their inputs here
so that the oracle and the GPU library see the same numbers.
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def fcc_lattice(n: int, rho: float, seed: int = 0, jitter: float = 0.0):
    """n atoms (n = 4 k^3) on an FCC lattice at number density rho in a cubic
    periodic box; optional Gaussian jitter (std `jitter`) from `seed`.
    Returns (positions [n][3] float64, box edge L)."""
    k = int(round((n / 4) ** (1.0 / 3.0)))
    if 4 * k ** 3 != n:
        raise ValueError("FCC needs n = 4 k^3")
    L = (n / rho) ** (1.0 / 3.0)
    a = L / k
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    g = np.stack(np.meshgrid(np.arange(k), np.arange(k), np.arange(k), indexing="ij"), -1).reshape(-1, 1, 3)
    x = ((g + basis[None]) * a).reshape(-1, 3) + 0.25 * a
    if jitter > 0:
        x = x + rng(seed).normal(scale=jitter, size=x.shape)
    return x.astype(np.float64), float(L)


def lattice(n: int, rho: float, seed: int = 0, jitter: float = 0.0):
    """n atoms on a cubic lattice at density rho: FCC when n = 4 k^3, simple
    cubic when n = k^3 (e.g. 4096 = 16^3), with optional Gaussian jitter.
    Returns (positions [n][3], box edge L)."""
    k4 = int(round((n / 4) ** (1.0 / 3.0)))
    if 4 * k4 ** 3 == n:
        return fcc_lattice(n, rho, seed, jitter)
    k = int(round(n ** (1.0 / 3.0)))
    if k ** 3 != n:
        raise ValueError("lattice needs n = 4 k^3 or k^3")
    L = (n / rho) ** (1.0 / 3.0)
    a = L / k
    g = np.stack(np.meshgrid(np.arange(k), np.arange(k), np.arange(k), indexing="ij"), -1).reshape(-1, 3)
    x = (g + 0.5) * a
    if jitter > 0:
        x = x + rng(seed).normal(scale=jitter, size=x.shape)
    return x.astype(np.float64), float(L)


def random_liquid(n: int, L: float, seed: int, min_dist: float = 0.9, max_tries: int = 200):
    """n points in a cubic periodic box of edge L drawn one by one from a
    seeded uniform distribution, rejecting any closer than min_dist to an
    accepted one (minimum image).  Used for small parity systems."""
    r = rng(seed)
    x = np.zeros((n, 3))
    m = 0
    while m < n:
        for _ in range(max_tries):
            p = r.uniform(0, L, 3)
            if m == 0:
                break
            d = x[:m] - p
            d -= L * np.rint(d / L)
            if np.min(np.einsum("ij,ij->i", d, d)) >= min_dist * min_dist:
                break
        else:
            raise RuntimeError("box too dense for random_liquid")
        x[m] = p
        m += 1
    return x


def permutation_subset(n: int, k: int, seed: int) -> np.ndarray:
    """The first k entries of a seeded permutation of range(n), int32."""
    return rng(seed).permutation(n)[:k].astype(np.int32)


def nearest_subset(x: np.ndarray, L: float, k: int, seed: int) -> np.ndarray:
    """Indices of the k atoms nearest (minimum image) to a seeded uniform
    centre in the box, sorted by index, int32."""
    c = rng(seed).uniform(0, L, 3)
    d = x - c
    if L > 0:
        d -= L * np.rint(d / L)
    order = np.argsort(np.einsum("ij,ij->i", d, d), kind="stable")[:k]
    return np.sort(order).astype(np.int32)


def uniform_points(P: int, lo, hi, seed: int) -> np.ndarray:
    """P points uniform in the box [lo, hi] (one entry per dimension)."""
    lo, hi = np.asarray(lo, float), np.asarray(hi, float)
    return rng(seed).uniform(lo, hi, size=(P, lo.size))


def uniform_hills(H: int, lo, hi, seed: int, w_range=(0.01, 1.0)) -> np.ndarray:
    """H hills [H][4] = (s_0, s_1, s_2, w): centres uniform in [lo, hi]
    (unused dimensions 0), heights uniform in w_range."""
    lo, hi = np.asarray(lo, float), np.asarray(hi, float)
    r = rng(seed)
    h = np.zeros((H, 4))
    h[:, : lo.size] = r.uniform(lo, hi, size=(H, lo.size))
    h[:, 3] = r.uniform(w_range[0], w_range[1], size=H)
    return h


def walk_hills(H: int, lo, hi, step, seed: int, w_range=(0.01, 1.0)) -> np.ndarray:
    """H hills whose centres follow a seeded reflected random walk in the CV
    box (per-dimension step std `step`), as a metadynamics run's deposits do;
    heights uniform in w_range."""
    lo, hi = np.asarray(lo, float), np.asarray(hi, float)
    step = np.broadcast_to(np.asarray(step, float), lo.shape)
    r = rng(seed)
    inc = r.normal(size=(H, lo.size)) * step
    s = np.empty((H, lo.size))
    cur = 0.5 * (lo + hi)
    span = hi - lo
    for k in range(H):
        cur = cur + inc[k]
        # reflect into [lo, hi]
        y = np.mod(cur - lo, 2 * span)
        cur = lo + np.where(y > span, 2 * span - y, y)
        s[k] = cur
    h = np.zeros((H, 4))
    h[:, : lo.size] = s
    h[:, 3] = r.uniform(w_range[0], w_range[1], size=H)
    return h


def chain_replicas(R: int, nbeads: int, seed: int, bond: float = 1.0, angle_deg: float = 109.47):
    """R chains of nbeads beads, bond length `bond`, bond angle `angle_deg`,
    torsions uniform in [-pi, pi) from `seed`; each chain starts at a seeded
    random point and orientation.  Returns positions [R*nbeads][3]."""
    r = rng(seed)
    th = np.deg2rad(angle_deg)
    out = np.zeros((R, nbeads, 3))
    for c in range(R):
        q, _ = np.linalg.qr(r.normal(size=(3, 3)))
        p = [np.zeros(3), np.array([bond, 0, 0]),
             np.array([bond - bond * np.cos(th), bond * np.sin(th), 0.0])]
        for i in range(3, nbeads):
            a, b, cc = p[i - 3], p[i - 2], p[i - 1]
            tor = r.uniform(-np.pi, np.pi)
            bc = cc - b
            bc /= np.linalg.norm(bc)
            nrm = np.cross(b - a, bc)
            nrm /= np.linalg.norm(nrm)
            m = np.array([bc, np.cross(nrm, bc), nrm]).T
            d2 = np.array([-bond * np.cos(th), bond * np.sin(th) * np.cos(tor), bond * np.sin(th) * np.sin(tor)])
            p.append(cc + m @ d2)
        out[c] = np.array(p[:nbeads]) @ q.T + r.uniform(-5, 5, 3)
    return out.reshape(-1, 3)


def log_uniform_sizes(W: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """W integers round(exp(U(ln lo, ln hi)))."""
    return np.rint(np.exp(rng(seed).uniform(np.log(lo), np.log(hi), size=W))).astype(np.int64)


def fcc_cluster(n: int, rho: float, seed: int):
    """n atoms: the n FCC sites (density rho) nearest a seeded point, i.e. a
    compact roughly spherical cluster, with a small seeded jitter."""
    r = rng(seed)
    k = int(np.ceil((2 * n) ** (1 / 3))) + 2
    x, L = fcc_lattice(4 * k ** 3, rho)
    c = np.full(3, L / 2) + r.uniform(-0.1, 0.1, 3)
    d = np.einsum("ij,ij->i", x - c, x - c)
    sel = x[np.argsort(d, kind="stable")[:n]] - c
    return sel + r.normal(scale=0.02, size=sel.shape)


def velocities(n: int, kT: float, mass: float, seed: int) -> np.ndarray:
    """Maxwell-Boltzmann velocities (std sqrt(kT/m)) from `seed`."""
    return rng(seed).normal(scale=np.sqrt(kT / mass), size=(n, 3))


def lj_clusters(W: int, lo: int, hi: int, rho: float, seed: int):
    """W compact LJ clusters (fcc_cluster) of log-uniform sizes in [lo, hi],
    concatenated walker after walker; returns (sizes, positions [sum n, 3])."""
    sizes = log_uniform_sizes(W, lo, hi, seed)
    x = np.concatenate([fcc_cluster(int(n), rho, seed=1000 * (seed + 1) + w) for w, n in enumerate(sizes)])
    return sizes, x


def native_pairs(x: np.ndarray, L: float, subset: np.ndarray, rcut: float) -> np.ndarray:
    """Pairs (i < j) of `subset` closer than rcut (minimum image, box L) in
    the configuration x, as a flat int32 array (i0, j0, i1, j1, ...)."""
    s = np.sort(np.asarray(subset))
    p = x[s]
    d = p[:, None, :] - p[None, :, :]
    d -= L * np.rint(d / L)
    r2 = (d ** 2).sum(-1)
    i, j = np.nonzero(np.triu(r2 < rcut * rcut, k=1))
    return np.stack([s[i], s[j]], axis=1).reshape(-1).astype(np.int32)
