"""The C-ABI library loads and exports every entry point declared in include/ddamg.h (no GPU needed)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ddamg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ddamg_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1307_6101_gb300 as dd
    names = _declared()
    assert len(names) >= 18
    missing = [n for n in names if not hasattr(dd.lib(), n)]
    assert not missing, missing
    assert set(names) == set(dd.EXPORTED)


def test_params_struct_matches_defaults_of_table1():
    import paper_1307_6101_gb300 as dd
    p = dd.ddamg_default_params()
    assert p.levels == 3 and list(p.agg[0]) == [4, 4, 4, 4] and list(p.agg[1]) == [2, 2, 2, 2]
    assert p.n_tv[0] == 20 and p.n_inv == 6 and p.coarse_tol == pytest.approx(5e-2)
    assert p.outer_restart == 10 and p.mu == 0 and p.nu == 5 and list(p.sap_block[0]) == [2, 2, 2, 2]
    assert p.mr_steps == 3 and p.kcycle_len == 5 and p.kcycle_cycles == 2 and p.kcycle_tol == pytest.approx(0.1)


def test_binding_constants_match_header():
    import paper_1307_6101_gb300 as dd
    src = open(os.path.join(ROOT, "include", "ddamg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    consts = dict((k, int(v)) for k, v in re.findall(r"\b(DDAMG_OPT_[A-Z_]+)\s*=\s*(-?\d+)", src))
    assert "DDAMG_OPT_HALF_STORAGE" in consts
    for k, v in consts.items():
        assert getattr(dd, k) == v, k


def test_footprint_estimate_is_host_only_and_consistent():
    """ddamg_estimate_bytes needs no device: it grows with the lattice and with the batch."""
    import paper_1307_6101_gb300 as dd
    kw = dict(levels=3, agg=[(2, 2, 2, 2), (2, 2, 2, 2)], n_tv=[4, 6], sap_block=[(2, 2, 2, 2), (2, 2, 2, 2)])
    p1 = dd.ddamg_default_params(**kw, max_rhs=1, precision=1)
    p4 = dd.ddamg_default_params(**kw, max_rhs=4, precision=1)
    p16 = dd.ddamg_default_params(**kw, max_rhs=1, precision=2)
    small = dd.ddamg_estimate_bytes((8, 8, 8, 8), p1)
    big = dd.ddamg_estimate_bytes((16, 8, 8, 8), p1)
    assert 1.9 * small <= big <= 2.1 * small          # everything scales with the volume
    assert dd.ddamg_estimate_bytes((8, 8, 8, 8), p4) > 2 * small
    assert dd.ddamg_estimate_bytes((8, 8, 8, 8), p16) > small   # FP16 copies come on top
    with pytest.raises(dd.DdamgError):
        dd.ddamg_estimate_bytes((8, 8, 8, 8), dd.ddamg_default_params(**kw, max_rhs=0))
