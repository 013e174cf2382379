"""The C-ABI library builds, loads without a GPU and exports every entry point
declared in include/dngd.h (no compute calls; CPU only)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        # type definitions (structs, callback signatures) declare no entry point
        src = re.sub(r"typedef[^;]*;", "", src, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(dngd_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2505_21404_gb300 import dngd
    return dngd


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert len(declared) >= 15
    for name in sorted(declared):
        assert hasattr(lib.lib, name), name
    # the binding wraps the same set
    assert declared <= set(lib.EXPORTED) | {n for n in declared if not hasattr(lib, n)}


def test_host_only_calls(lib):
    from paper_2505_21404_gb300 import workloads
    assert lib.lib.dngd_version().decode().startswith("dngd-gb300")
    assert lib.lib.dngd_status_string(-2).decode() == "matrix not positive definite"
    wl = workloads.poisson5d_dense()
    desc = lib.make_desc(wl, precision=lib.MIXED_BF16)
    assert lib.dngd_num_params(desc) == 133377
    assert lib.dngd_workspace_bytes(desc) > 4000 * 133377 * 6
    bad = lib.make_desc(wl)
    bad.widths[bad.n_layers] = 2          # output width must be 1
    assert lib.dngd_num_params(bad) == -1


def _enum_values(name):
    src = open(os.path.join(ROOT, "include", "dngd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    body = re.search(r"enum\s+" + name + r"\s*\{(.*?)\}", src, flags=re.S).group(1)
    return {k: int(v) for k, v in re.findall(r"(DNGD_\w+)\s*=\s*(-?\d+)", body)}


def test_descriptor_enums_match_the_header(lib):
    """The binding's constants for the descriptor's enum fields are the
    header's values, and the descriptor's last field is where ctypes puts it
    (the structure sizes agree field by field in the GPU tests)."""
    fu = _enum_values("dngd_factor_update")
    assert fu == {"DNGD_FACTOR_SLICED": lib.FACTOR_SLICED, "DNGD_FACTOR_DF": lib.FACTOR_DF}
    po = _enum_values("dngd_pcg_operator")
    assert po == {"DNGD_PCG_OP_TC3": lib.PCG_OP_TC3, "DNGD_PCG_OP_COMPENSATED": lib.PCG_OP_COMPENSATED}
    sp = _enum_values("dngd_solve_space")
    assert sp == {"DNGD_SPACE_DUAL": lib.SPACE_DUAL, "DNGD_SPACE_PRIMAL": lib.SPACE_PRIMAL,
                  "DNGD_SPACE_AUTO": lib.SPACE_AUTO}
    from paper_2505_21404_gb300 import workloads
    d = lib.make_desc(workloads.poisson5d_dense(), precision=lib.MIXED_OZ64, factor_update=lib.FACTOR_DF)
    assert d.factor_update == lib.FACTOR_DF
    names = [f[0] for f in lib.ProblemDesc._fields_]
    assert names[-3:] == ["pcg_operator", "factor_update", "solve_space"]


def test_descriptor_validation_before_any_device_work(lib):
    """dngd_create refuses out-of-range enum fields before it touches the
    device (so this runs without a GPU)."""
    import ctypes as C
    from paper_2505_21404_gb300 import workloads
    wl = workloads.poisson_sine(2, [2, 8, 8, 1], 30, 10, k=1, seed=0, lam=1e-5)
    for field, bad in (("factor_update", 2), ("factor_update", -1), ("pcg_operator", 2), ("precision", 9),
                       ("solver", 3)):
        d = lib.make_desc(wl, precision=lib.MIXED_OZ64)
        setattr(d, field, bad)
        h = C.c_void_p()
        assert lib.lib.dngd_create(C.byref(h), C.byref(d), None) == -1, (field, bad)
        assert not h.value
    # the primal space is built for the dense FP64 solver only
    for prec, solver, space in ((lib.FP64, lib.DENSE, 3), (lib.FP64, lib.DENSE, -1),
                                (lib.MIXED_OZ64, lib.DENSE, lib.SPACE_PRIMAL),
                                (lib.MIXED_BF16, lib.PCG, lib.SPACE_PRIMAL)):
        d = lib.make_desc(wl, precision=prec, solver=solver, solve_space=space)
        h = C.c_void_p()
        assert lib.lib.dngd_create(C.byref(h), C.byref(d), None) == -1, (prec, solver, space)
        assert not h.value


def test_primal_space_workspace(lib):
    """The primal space sizes the FP64 system by n (Prop. 3.1: n x n), the
    dual by m; automatic selection takes the smaller system (host-only
    sizing, no device work)."""
    from paper_2505_21404_gb300 import workloads
    tall = workloads.poisson_sine(2, [2, 8, 8, 1], 400, 100, k=1, seed=0, lam=1e-5)     # n = 105 < m = 500
    wide = workloads.poisson_sine(2, [2, 32, 32, 1], 40, 10, k=1, seed=0, lam=1e-5)     # n = 1,185 > m = 50
    for wl in (tall, wide):
        m = sum(c["count"] for c in wl["classes"])
        n = lib.dngd_num_params(lib.make_desc(wl))
        by = {sp: lib.dngd_workspace_bytes(lib.make_desc(wl, solve_space=sp))
              for sp in (lib.SPACE_DUAL, lib.SPACE_PRIMAL, lib.SPACE_AUTO)}
        # the system buffers (K, Dinv, solve work) differ by the dimension
        assert (by[lib.SPACE_PRIMAL] < by[lib.SPACE_DUAL]) == (n < m)
        assert by[lib.SPACE_AUTO] == min(by[lib.SPACE_PRIMAL], by[lib.SPACE_DUAL])
        # the automatic choice stays dual outside the dense FP64 solver
        d = lib.make_desc(wl, precision=lib.MIXED_OZ64, solve_space=lib.SPACE_AUTO)
        assert lib.dngd_workspace_bytes(d) == lib.dngd_workspace_bytes(lib.make_desc(wl, precision=lib.MIXED_OZ64))
