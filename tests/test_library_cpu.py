"""CPU-side checks of the C ABI library: it builds for sm_103a, loads, and
exports every function declared in include/bie.h (no compute calls here)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    with open(os.path.join(ROOT, "include", "bie.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(bie_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def built_lib():
    from paper_2108_01786_gb300 import _build
    _build.build()
    import paper_2108_01786_gb300 as P
    return P.lib()


def test_header_declares_expected_entry_points():
    names = _header_functions()
    for n in ["bie_create", "bie_destroy", "bie_last_error", "bie_set_geometry", "bie_set_flow",
              "bie_assemble", "bie_solve", "bie_normal_velocity", "bie_rhs", "bie_matvec",
              "bie_sample_entries", "bie_solve_host", "bie_default_opts"]:
        assert n in names


def test_library_exports_every_header_symbol(built_lib):
    for n in _header_functions():
        assert hasattr(built_lib, n), n


def test_binding_covers_header(built_lib):
    import paper_2108_01786_gb300 as P
    for n in _header_functions():
        assert n in P.SIGNATURES, n
        assert callable(getattr(P, n)), n


def test_default_opts_and_null_handling(built_lib):
    """Host-only calls: defaults, and NULL-argument errors that never touch a GPU."""
    import ctypes
    import paper_2108_01786_gb300 as P
    o = P.bie_default_opts()
    assert o.rtol == 1e-14 and o.restart == 50 and o.row_flip == 1 and o.x0 == 0
    assert P.bie_default_opts(x0=1).x0 == 1
    import pytest
    with pytest.raises(TypeError):
        P.bie_default_opts(initial_guess=1)
    assert built_lib.bie_last_error(None) == b"null context"
    assert built_lib.bie_set_flow(None, 1.0, None) == P.BIE_ERR_ARG
    assert built_lib.bie_assemble(None, 0) == P.BIE_ERR_ARG
    assert built_lib.bie_create(None, 0, None) == P.BIE_ERR_ARG
    built_lib.bie_destroy(None)


def test_no_oracle_in_product_path():
    """The product package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_2108_01786_gb300")
    for dp, _, fs in os.walk(pkg):
        for fn in fs:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                with open(os.path.join(dp, fn)) as f:
                    src = f.read()
                assert "import oracle" not in src and "from oracle" not in src, fn


def test_save_and_load_state_roundtrip(tmp_path):
    import numpy as np
    import workloads as W
    import paper_2108_01786_gb300 as P
    g, f, ph = W.one_ellipse_640()
    om = np.random.default_rng(0).standard_normal(g.N)
    p = tmp_path / "state.npz"
    P.save_state(p, g, f, ph, omega=om, t=np.float64(0.25))
    d = P.load_state(p)
    assert list(d["M"]) == list(g.M) and np.array_equal(d["zeta"], g.zeta)
    assert np.array_equal(d["phit"], ph) and np.array_equal(d["omega"], om)
    assert float(d["V1"]) == f.V1 and np.array_equal(d["a"], f.a) and float(d["t"]) == 0.25


def test_static_limit_matches_header():
    """The binding's STATIC_MAXN is the header's BIE_STATIC_MAXN."""
    import paper_2108_01786_gb300 as P
    with open(os.path.join(ROOT, "include", "bie.h")) as f:
        m = re.search(r"#define\s+BIE_STATIC_MAXN\s+(\d+)", f.read())
    assert m and int(m.group(1)) == P.STATIC_MAXN
