"""The C-ABI library builds, loads and exports every symbol declared in include/natconv.h.

These tests make no compute call (they run on CPU-only machines)."""

import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1904_00182_gb300 import build
    build.build()
    from paper_1904_00182_gb300 import _abi
    return _abi.load_library()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "natconv.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nc_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert len(names) >= 16
    for name in names:
        assert hasattr(lib, name), name
    from paper_1904_00182_gb300 import _abi
    assert sorted(_abi.EXPORTS) == names


def test_default_params_and_footprint(lib):
    from paper_1904_00182_gb300 import Grid, default_params, footprint_bytes
    p = default_params()
    assert p.alpha == 1e3 and p.k_s == 100.0 and p.q_c == pytest.approx(8.81)
    assert p.newton_rtol == 1e-8 and p.restart == 30
    from paper_1904_00182_gb300 import NC_ARITH_FP64, NC_BASIS_FP64, NC_PREC_MIXED
    assert p.precision == NC_PREC_MIXED and p.outer_arith == NC_ARITH_FP64 and p.krylov_basis == NC_BASIS_FP64
    b16 = footprint_bytes(Grid(16, 16, 16, 1 / 16), p)
    b32 = footprint_bytes(Grid(32, 32, 32, 1 / 32), p)
    assert 0 < b16 < b32
    # 128^3 mixed fits easily in the 288 GB of one GB300
    assert footprint_bytes(Grid(128, 128, 128, 1 / 128), p) < 8e9


def test_invalid_arguments_are_rejected_without_a_device(lib):
    from paper_1904_00182_gb300 import Grid, NatConvError, default_params, footprint_bytes
    p = default_params()
    with pytest.raises(NatConvError) as e:
        footprint_bytes(Grid(15, 16, 16, 1 / 16), p)          # odd: no multigrid hierarchy
    assert e.value.status_name == "NC_ERR_ARG"
    with pytest.raises(NatConvError):
        footprint_bytes(Grid(16, 16, 16, -1.0), p)
    p.heated_layers = 16
    with pytest.raises(NatConvError):
        footprint_bytes(Grid(16, 16, 16, 1 / 16), p)
    assert lib.nc_last_error(None)
    p = default_params()
    p.restart = 0
    with pytest.raises(NatConvError):
        footprint_bytes(Grid(16, 16, 16, 1 / 16), p)
    p = default_params()
    p.outer_arith = 2
    with pytest.raises(NatConvError):
        footprint_bytes(Grid(16, 16, 16, 1 / 16), p)
    p = default_params()
    p.krylov_basis = 2
    with pytest.raises(NatConvError):
        footprint_bytes(Grid(16, 16, 16, 1 / 16), p)
    p = default_params()
    p.mg_smoother = 2
    with pytest.raises(NatConvError):
        footprint_bytes(Grid(16, 16, 16, 1 / 16), p)
    p = default_params()
    p.mg_smoother, p.mg_tail_nodes = 1, 4096          # the fused tail smooths with block Jacobi
    with pytest.raises(NatConvError):
        footprint_bytes(Grid(16, 16, 16, 1 / 16), p)
    p.mg_tail_nodes = 0
    # the z-line factors: 24 values per node on the levels between the finest and the coarsest
    assert footprint_bytes(Grid(16, 16, 16, 1 / 16), p) > footprint_bytes(Grid(16, 16, 16, 1 / 16), default_params())


def _struct_fields(name):
    """Field names, in order, of the typedef struct `name` in the header."""
    text = open(os.path.join(ROOT, "include", "natconv.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    m = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + ";", text)
    assert m, name
    names = []
    for decl in m.group(1).split(";"):
        decl = decl.strip()
        if not decl:
            continue
        parts = decl.split(None, 1)
        if parts[0] in ("long", "unsigned"):
            parts = parts[1].split(None, 1)
        for v in parts[1].split(","):
            names.append(re.sub(r"\[.*\]", "", v).strip().lstrip("*"))
    return names


@pytest.mark.parametrize("cname, pyname", [("nc_params", "Params"), ("nc_stats", "Stats"), ("nc_grid", "Grid")])
def test_python_structures_mirror_the_header(cname, pyname):
    from paper_1904_00182_gb300 import _abi
    assert [f for f, _ in getattr(_abi, pyname)._fields_] == _struct_fields(cname)


def test_product_has_no_cpu_fallback():
    """The package never imports the oracle and raises when the library is missing."""
    pkg = os.path.join(ROOT, "paper_1904_00182_gb300")
    for f in os.listdir(pkg):
        if f.endswith(".py"):
            src = open(os.path.join(pkg, f)).read()
            assert "import oracle" not in src and "from oracle" not in src, f
    from paper_1904_00182_gb300 import _abi
    with pytest.raises(ImportError):
        _abi.load_library(os.path.join(ROOT, "does_not_exist.so"))


def test_torch_design_recipe_matches_numpy_recipe():
    """The device-side design generator follows the same recipe as the NumPy one: given the same
    normals it gives the same smoothed field and the requested volume fraction."""
    import torch
    from synthetic import designs
    rng = np.random.default_rng(5)
    noise = rng.standard_normal((6, 5, 7))
    a = designs._cone_smooth(noise, 1.5)
    a = (a - a.min()) / (a.max() - a.min())
    b = designs.filtered_random_torch(7, 5, 6, seed=0, noise=noise).numpy()
    assert np.abs(a.ravel() - b).max() < 1e-14
    c = designs.filtered_random_torch(12, 12, 12, seed=3, volfrac=0.2).numpy()
    assert abs(c.mean() - 0.2) < 1e-6 and c.min() >= 0.0 and c.max() <= 1.0
    d = designs.filtered_random_torch(12, 12, 12, seed=3, volfrac=0.2).numpy()
    assert np.array_equal(c, d)


def test_solver_presets_by_alpha():
    """The z-line smoother with omega 0.7 from alpha = 1e6 on, the library defaults below; the preset's
    fields are nc_params fields and the combination validates (no fused tail)."""
    from paper_1904_00182_gb300 import Grid, NC_SMOOTH_ZLINE, default_params, footprint_bytes
    from paper_1904_00182_gb300.presets import solver_settings
    assert solver_settings(1e3) == {} and solver_settings(9.9e5) == {}
    s = solver_settings(1e6)
    assert s == {"mg_smoother": NC_SMOOTH_ZLINE, "omega": 0.7}
    p = default_params(alpha=1e6, **s)
    assert p.mg_smoother == NC_SMOOTH_ZLINE and p.omega == 0.7 and p.mg_tail_nodes == 0
    assert footprint_bytes(Grid(16, 16, 32, 1 / 32), p) > 0
