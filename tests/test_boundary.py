"""The C-ABI library loads, exports every symbol include/bp.h declares and
rejects a null context at every entry point (no compute calls: runs without a
GPU)."""
import ctypes
import os

import pytest

from paper_2208_08038_gb300 import binding, build_lib


@pytest.fixture(scope="module")
def libpath():
    return build_lib.build()


def test_header_declares_the_api():
    names = binding.header_functions()
    for f in ["bp_create", "bp_destroy", "bp_add_species", "bp_load_particles", "bp_set_medium",
              "bp_add_laser", "bp_add_probe", "bp_step", "bp_sync", "bp_read_field", "bp_write_field",
              "bp_read_probe", "bp_read_particles", "bp_residual", "bp_last_error"]:
        assert f in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [f for f in binding.header_functions() if not hasattr(L, f)]
    assert not missing, missing


def test_library_is_built_for_sm103a_only():
    """Every translation unit is compiled with one -gencode, for sm_103a, and
    no other architecture flag."""
    assert build_lib.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    flat = " ".join(build_lib.FLAGS)
    assert "-arch" not in flat and "-gencode" not in flat and "compute_" not in flat


def test_binding_signatures_cover_header():
    assert set(binding.header_functions()) <= set(binding._SIGS)


def test_oracle_not_imported_by_product():
    """The product package never imports the oracle."""
    pkg = os.path.dirname(binding.__file__)
    for root, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(root, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt and "bp_oracle" not in txt, f


def test_entry_points_reject_a_null_context(libpath):
    """Every entry point that takes a context checks it before any CUDA call:
    a null context gives BP_ERR_ARG (and no crash), so this runs without a GPU."""
    L = binding.lib()
    err_arg = -1
    zero = {ctypes.c_int: 0, ctypes.c_int64: 0, ctypes.c_uint64: 0, ctypes.c_double: 0.0}
    checked = 0
    for name, (res, args) in binding._SIGS.items():
        f = getattr(L, name)
        vals = [zero.get(a, None) for a in args]
        if name == "bp_destroy":
            f(None)
            continue
        out = f(*vals)
        if name == "bp_last_error":
            assert out == b"null context"
        elif name == "bp_kernel_launches":
            assert out == 0
        else:
            assert out == err_arg, name
            checked += 1
    assert checked >= 25


def _grid(dims, n, dx, dt, tile=(0, 0, 0), boundary=(0, 0, 0)):
    g = binding.GridDesc()
    g.dims = dims
    for a in range(3):
        g.n[a] = n[a] if a < len(n) else 1
        g.dx[a] = dx[a] if a < len(dx) else 1.0
        g.boundary[a] = boundary[a]
        g.tile[a] = tile[a]
    g.dt = dt
    g.deposit_mode = binding.BP_DEPOSIT_SORTED
    return g


@pytest.mark.parametrize("desc, code", [
    (_grid(0, (64,), (1.0,), 0.5), binding.BP_ERR_ARG),                        # no such dimension
    (_grid(4, (64,) * 3, (1.0,) * 3, 0.5), binding.BP_ERR_ARG),
    (_grid(1, (3,), (1.0,), 0.5), binding.BP_ERR_ARG),                         # fewer than 4 cells
    (_grid(1, (64,), (0.0,), 0.5), binding.BP_ERR_ARG),                        # zero cell size
    (_grid(1, (24,), (1.0,), 0.5), binding.BP_ERR_ARG),                        # not whole 16-cell tiles
    (_grid(2, (64, 64), (1.0, 1.0), 0.5, tile=(8, 16, 0)), binding.BP_ERR_ARG),  # a tile other than 16 x 16
    (_grid(1, (64,), (1.0,), 0.0), binding.BP_ERR_CFL),                        # dt = 0
    (_grid(1, (64,), (1.0,), 1.0), binding.BP_ERR_CFL),                        # c dt = dx
    (_grid(2, (64, 64), (1.0, 1.0), 0.75), binding.BP_ERR_CFL),                # 0.75 sqrt(2) > 1
    (_grid(3, (2048, 1024, 1024), (1.0,) * 3, 0.5), binding.BP_ERR_ARG),      # 2^31 cells
    (_grid(3, (1032, 1032, 1032), (1.0,) * 3, 0.5), binding.BP_ERR_ARG),      # cell index needs 33 bits
])
def test_create_rejects_a_bad_grid_before_any_cuda_call(libpath, desc, code):
    """bp_create checks the grid description (dimensions, sizes, tile shape,
    the Courant limit c dt sqrt(sum 1/dx^2) < 1 of the Yee scheme, the 31-bit
    cell index) before it touches the device, so these run without a GPU."""
    L = binding.lib()
    out = ctypes.c_void_p(1234)
    rc = L.bp_create(ctypes.byref(desc), None, None, ctypes.byref(out))
    assert rc == code
    assert out.value is None  # *out is cleared and set only on BP_OK


def test_create_rejects_null_pointers(libpath):
    L = binding.lib()
    out = ctypes.c_void_p()
    g = _grid(1, (64,), (1.0,), 0.5)
    assert L.bp_create(None, None, None, ctypes.byref(out)) == binding.BP_ERR_ARG
    assert L.bp_create(ctypes.byref(g), None, None, None) == binding.BP_ERR_ARG


def test_binding_refuses_to_run_without_the_library(monkeypatch, tmp_path):
    """No fallback: with the library missing the binding raises."""
    monkeypatch.setattr(binding, "_lib", None)
    monkeypatch.setattr(binding, "LIB_PATH", str(tmp_path / "libbp.so"))
    with pytest.raises(RuntimeError, match="CUDA library missing"):
        binding.lib()
