"""The five workloads as data (paper_2301_04835_b300/configs.json) agree with
what bench.py and the tests run, so the file a user reads is the one that is
measured."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _cfg():
    sys.path.insert(0, ROOT)
    import paper_2301_04835_b300 as wt  # loads without a GPU; no kernel is called

    return wt.load_config()


def test_five_workloads_present():
    cfg = _cfg()
    assert set(cfg) == {"mueller_brown", "lj4096", "chain1024", "walkers256", "surrogate32768"}
    for c in cfg.values():
        assert c["precision"] in ("f32", "f64") and len(c["sigma"]) == len(c["cvs"])


def test_bench_constants_match_the_configs():
    sys.path.insert(0, ROOT)
    import bench

    cfg = _cfg()
    lj = cfg["lj4096"]
    assert (bench.N_ATOMS, bench.RHO, bench.N_TAG, bench.N_RG, bench.H_PRE) == (
        lj["walker_sizes"][0], lj["rho"], lj["n_tag"], lj["n_rg"], lj["hills"])
    assert tuple(bench.SIGMA) == tuple(lj["sigma"])
    wk = cfg["walkers256"]
    assert (bench.W_CL, bench.CL_LO, bench.CL_HI, bench.H_CL) == (wk["walkers"], wk["size_lo"], wk["size_hi"],
                                                                 wk["hills"])
    assert tuple(bench.CL_SIGMA) == tuple(wk["sigma"])
    su = cfg["surrogate32768"]
    assert (bench.N_SU, bench.H_SU) == (su["walker_sizes"][0], su["hills"])
    assert tuple(bench.SU_SIGMA) == tuple(su["sigma"])
    mb = cfg["mueller_brown"]
    assert bench.MB_STEPS == mb["steps"] and tuple(bench.MB_BINS) == tuple(mb["grid"][0])
    assert tuple(bench.MB_LO) == tuple(mb["grid"][1]) and tuple(bench.MB_HI) == tuple(mb["grid"][2])
    assert mb["steps"] // mb["stride"] == mb["hills"]


def test_chain_config_matches_the_adjoint_workload():
    cfg = _cfg()["chain1024"]
    assert [c["a"] for c in cfg["cvs"]] == [[5, 7, 9, 15], [7, 9, 15, 17]]
    assert all(c["period"] == pytest.approx(2 * np.pi) for c in cfg["cvs"])
