"""Builders that set up the same seeded system for the oracle and for the GPU
library (test helper; the two sides share only the inputs from `synth`)."""
from __future__ import annotations

import numpy as np

import synth

KIND = {"component": 1, "dihedral": 2, "coordination": 3, "rg": 4, "qpairs": 5, "distance": 6, "angle": 7,
        "gyration": 8}


def oracle_system(spec):
    import oracle as o

    cvs = [o.CV(KIND[c["kind"]], a=c.get("a"), b=c.get("b"), axis=c.get("axis", 0), r0=c.get("r0", 1.5),
                nn=c.get("nn", 6), mm=c.get("mm", 12), scale=c.get("scale", 0.0), flags=c.get("flags", 0),
                period=c.get("period", 0.0)) for c in spec["cvs"]]
    grid = spec.get("grid")
    kw = dict(engine={"none": 0, "mb": 1, "lj": 2, "chain": 3, "wells3": 5}[spec.get("engine", "none")],
              walker_n=list(spec["walker_sizes"]), cvs=cvs, dims=spec.get("dims", 3), box=tuple(spec.get("box", (0, 0, 0))),
              dt=spec.get("dt", 1e-3), friction=spec.get("friction", 1.0), mass=spec.get("mass", 1.0),
              kT=spec.get("kT", 1.0), seed=spec.get("seed", 0), sigma=tuple(spec["sigma"]), w0=spec.get("w0", 1.0),
              gamma=spec.get("gamma", 10.0), stride=spec.get("stride", 100), hill_cap=spec.get("capacity", 1000))
    if grid:
        kw.update(grid_bins=tuple(grid[0]), grid_lo=tuple(grid[1]), grid_hi=tuple(grid[2]))
    if spec.get("bias_grid"):
        kw.update(bias_grid=True)
    return o.System(**kw)


def gpu_handle(spec, precision):
    import paper_2301_04835_b300 as wt

    m = wt.Wtmd(precision=precision, sigma=spec["sigma"], w0=spec.get("w0", 1.0), gamma=spec.get("gamma", 10.0),
                kT=spec.get("kT", 1.0), stride=spec.get("stride", 100), capacity=spec.get("capacity", 1000),
                seed=spec.get("seed", 0), grid=spec.get("grid"), engine=spec.get("engine", "none"),
                dims=spec.get("dims", 0), walker_sizes=spec["walker_sizes"], dt=spec.get("dt", 1e-3),
                friction=spec.get("friction", 1.0), mass=spec.get("mass", 1.0), box=tuple(spec.get("box", (0, 0, 0))))
    for c in spec["cvs"]:
        m.cv_define(KIND[c["kind"]], a=c.get("a"), b=c.get("b"), axis=c.get("axis", 0), r0=c.get("r0", 1.5),
                    nn=c.get("nn", 6), mm=c.get("mm", 12), scale=c.get("scale", 0.0), flags=c.get("flags", 0),
                    period=c.get("period", 0.0))
    if spec.get("bias_grid"):
        m.bias_source(wt.BIAS_GRID)
    return m


def lj_fluid_spec(n=4096, rho=0.8, n_tag=512, n_rg=64, seed=0, jitter=0.05, capacity=200000):
    """LJ fluid at rho* = 0.8, T* = 1 with the two CVs of the 4096-atom
    workload: mean coordination of tagged atoms (r0 = 1.5, n = 6, m = 12) and
    Rg of the atoms nearest a seeded centre."""
    x, L = synth.lattice(n, rho, seed=seed, jitter=jitter)
    tag = synth.permutation_subset(n, n_tag, seed + 1)
    rg = synth.nearest_subset(x, L, n_rg, seed + 2)
    spec = dict(engine="lj", walker_sizes=[n], box=(L, L, L), dt=0.005, kT=1.0, friction=1.0,
                sigma=(0.05, 0.1), gamma=8.0, w0=1.0, stride=100, capacity=capacity,
                cvs=[dict(kind="coordination", a=tag, r0=1.5, nn=6, mm=12), dict(kind="rg", a=rg)])
    return spec, x, L


def to_np(t):
    return t.detach().cpu().double().numpy()
