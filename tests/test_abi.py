"""The C ABI library loads and exports every function include/gpcg.h
declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "gpcg.h")).read()
    return sorted(set(re.findall(r"GPCG_API\s+[\w\s\*]+?\b(gpcg_\w+)\s*\(", src)))


def test_header_declares_the_api():
    names = declared()
    for required in ("gpcg_create", "gpcg_base_solve", "gpcg_n1_screen", "gpcg_destroy",
                     "gpcg_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1803_03290_gb300 import binding
    lib = binding.load()
    for name in declared():
        assert hasattr(lib, name), name
    assert set(binding.EXPORTS) <= set(declared())


def test_invalid_arguments_fail_before_the_gpu():
    import numpy as np
    from paper_1803_03290_gb300 import binding
    from gridgen import config_grid
    g = config_grid("grid120")
    bad = g.copy()
    bad.bus_type = bad.bus_type.copy()
    bad.bus_type[:] = 0           # no slack
    with pytest.raises(binding.GPCGError) as e:
        binding.GPCG(bad)
    assert e.value.status == 1 and "slack" in str(e.value)
    bad = g.copy()
    bad.x = bad.x.copy()
    bad.x[3] = 0.0
    with pytest.raises(binding.GPCGError) as e:
        binding.GPCG(bad)
    assert e.value.status == 1
    bad = g.copy()
    bad.f = bad.f.copy()
    bad.f[0] = bad.t[0]
    with pytest.raises(binding.GPCGError) as e:
        binding.GPCG(bad)
    assert e.value.status == 1
    for v in (-1.0, 0.0, float("nan")):
        bad = g.copy()
        bad.tap = np.ones(g.n_branch)
        bad.tap[5] = v
        with pytest.raises(binding.GPCGError) as e:
            binding.GPCG(bad)
        assert e.value.status == 1 and "turns ratio" in str(e.value)
    pv = int(np.flatnonzero(g.bus_type == 1)[0])
    bad = g.copy()
    bad.Q_max = np.ones(g.n_bus)               # Q_max without Q_min
    with pytest.raises(binding.GPCGError) as e:
        binding.GPCG(bad)
    assert e.value.status == 1 and "Q_min and Q_max" in str(e.value)
    bad.Q_min = np.zeros(g.n_bus)
    bad.Q_min[pv] = 2.0                        # an empty interval at a PV bus
    with pytest.raises(binding.GPCGError) as e:
        binding.GPCG(bad)
    assert e.value.status == 1 and "reactive limits" in str(e.value)
    with pytest.raises(binding.GPCGError):
        binding.default_options(precision=7) and binding.GPCG(g, precision=7)


def _struct_fields(name):
    src = open(os.path.join(ROOT, "include", "gpcg.h")).read()
    body = re.search(r"typedef struct \{([^}]*)\}\s*" + name + ";", src).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    out = []
    for decl in body.split(";"):
        decl = decl.strip()
        if decl:
            out += [v.strip().lstrip("*") for v in decl.split(None, 1)[1].split(",")]
    return out


def test_binding_structs_follow_the_header():
    from paper_1803_03290_gb300 import binding
    assert [k for k, _ in binding.Options._fields_] == _struct_fields("gpcg_options")
    assert [k for k, _ in binding.Info._fields_] == _struct_fields("gpcg_info")
    src = open(os.path.join(ROOT, "include", "gpcg.h")).read()
    assert int(re.search(r"#define GPCG_MAX_TAIL_ROWS (\d+)", src).group(1)) == binding.MAX_TAIL_ROWS
    assert int(re.search(r"#define GPCG_MAX_EXT_ROWS (\d+)", src).group(1)) == binding.MAX_EXT_ROWS


@pytest.mark.parametrize("bad", [dict(tail_rows=-2), dict(tail_rows=249), dict(tile=3),
                                 dict(ctas_per_sm=-1), dict(wait_limit=-1)])
def test_bad_options_fail_before_the_gpu(bad):
    from paper_1803_03290_gb300 import binding
    from gridgen import config_grid
    with pytest.raises(binding.GPCGError) as e:
        binding.GPCG(config_grid("grid120"), **bad)
    assert e.value.status == 1
