"""CPU checks of the C ABI: the library builds, loads, and exports every
function include/ok.h declares; option defaults and host-side argument
validation work without a GPU (no compute call is made here)."""
import ctypes
import os
import re

import pytest

import paper_1603_04570_gb300 as ok

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(ok_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["ok_grid_create", "ok_grid_destroy", "ok_assemble_rhs", "ok_newton_step",
                     "ok_timestep", "ok_solve_batch", "ok_init_w", "ok_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = ok.load()
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
    assert ok.version().startswith("ok-gb300")


def test_default_opts_match_header_documentation():
    o = ok.ok_default_opts()
    assert (o.restart, o.q_A, o.n_V, o.k_R, o.smooth_pre, o.smooth_post) == (30, 10, 5, 1, 2, 2)
    assert o.precision == ok.OK_FP64 and o.gmres_rtol == 1e-10 and o.smooth_lo_frac == 0.25
    assert o.use_graphs == 1 and o.fuse_coarse == 1
    assert o.tile_fine == 1 and o.use_pdl == 1 and o.reorth == 1
    assert ok.Opts.gmres_rtol.offset == 64 and ctypes.sizeof(ok.Opts) == 96   # 16 ints, 4 doubles


@pytest.mark.parametrize("dim,n,kw,msg", [
    (4, 8, {}, "dim"),
    (2, 1, {}, "n must"),
    (2, 8, {"restart": 0}, "restart"),
    (2, 8, {"restart": 64}, "restart"),
    (2, 8, {"k_R": 3}, "k_R"),
    (2, 8, {"precision": 7}, "precision"),
    (2, 8, {"q_A": 0}, "q_A"),
    (2, 8, {"gmres_rtol": 0.0}, "tolerances"),
    (2, 8, {"tile_fine": 4}, "tile_fine"),
    (2, 8, {"reorth": 3}, "reorth"),
])
def test_invalid_arguments_rejected_on_host(dim, n, kw, msg):
    p = ok.Params(0.04, 100.0, 0.0, 1.0, 1e-4)
    with pytest.raises(ok.OkError) as e:
        ok.ok_grid_create(dim, n, p, ok.ok_default_opts(**kw))
    assert e.value.status == ok.OK_ERR_INVALID_ARG and msg in str(e.value)


def test_invalid_params_rejected_on_host():
    for bad in [ok.Params(0.0, 100, 0, 1, 1e-4), ok.Params(0.04, 100, 0, 0.0, 1e-4),
                ok.Params(0.04, 100, 0, 1, -1.0), ok.Params(0.04, -1, 0, 1, 1e-4)]:
        with pytest.raises(ok.OkError) as e:
            ok.ok_grid_create(2, 8, bad)
        assert e.value.status == ok.OK_ERR_INVALID_ARG


def test_large_odd_coarse_level_is_accepted():
    """A coarsest level above the dense-inverse limit (18^3 unknowns for 3D
    n = 17) is solved by Chebyshev iteration, so argument validation accepts
    it (without a GPU the call gets as far as its first CUDA call)."""
    try:
        h = ok.ok_grid_create(3, 17, ok.Params(0.04, 100, 0, 1, 1e-4))
    except ok.OkError as e:
        assert e.status != ok.OK_ERR_INVALID_ARG, str(e)
    else:
        ok.ok_grid_destroy(h)


def test_status_codes_match_the_header():
    text = open(os.path.join(ROOT, "include", "ok.h")).read()
    codes = dict((name, int(v)) for name, v in re.findall(r"^\s*(OK_(?:SUCCESS|ERR_\w+))\s*=\s*(\d+)", text, re.M))
    assert codes == {name: code for code, name in ok.STATUS_NAMES.items()}
    assert ok.OK_ERR_INTERNAL == 7


def test_serving_structs_match_the_header():
    assert ctypes.sizeof(ok.ServeRequest) == 224 and ok.ServeRequest.arrival.offset == 80
    assert ok.ServeRequest.device_bytes.offset == 120
    assert ctypes.sizeof(ok.ServeInfo) == 40 and ok.ServeInfo.seconds.offset == 24
    assert ok.ServeInfo.peak_cohort.offset == 32 and ok.ServeInfo.cohort_steps.offset == 36


def test_serve_rejects_invalid_arguments_on_host():
    st, _, _ = ok.ok_serve([], max_inflight=0, mem_budget=1 << 30)
    assert st == ok.OK_ERR_INVALID_ARG


def test_binding_rejects_badly_typed_arrays():
    """Argument marshalling: float64, contiguous, of the stated size."""
    import numpy as np
    assert ok._ptr(None) is None
    a = np.zeros(8)
    assert ok._ptr(a, 8) == a.ctypes.data
    with pytest.raises(TypeError):
        ok._ptr(np.zeros(8, dtype=np.float32), 8, "u")
    with pytest.raises(TypeError):
        ok._ptr(np.zeros(16)[::2], 8, "u")                      # not contiguous
    with pytest.raises(ValueError):
        ok._ptr(np.zeros(7), 8, "u")
    with pytest.raises(TypeError):
        ok._ptr([0.0] * 8, 8, "u")
    torch = pytest.importorskip("torch")
    t = torch.zeros(8, dtype=torch.float64)
    assert ok._ptr(t, 8) == t.data_ptr()
    with pytest.raises(TypeError):
        ok._ptr(torch.zeros(8, dtype=torch.float32), 8, "u")
    with pytest.raises(ValueError):
        ok._ptr(torch.zeros(9, dtype=torch.float64), 8, "u")


def test_host_diagnostic_wrappers_validate_shapes():
    import numpy as np
    with pytest.raises(ValueError):
        ok.ok_hessenberg_eigenvalues(np.zeros((3, 4)))
    with pytest.raises(ValueError):
        ok.ok_givens_unrotate(np.zeros((3, 3)), np.zeros(3), np.zeros(3))   # R must be (k+1) x k
    assert ok.ok_givens_unrotate(np.zeros((1, 0)), np.zeros(0), np.zeros(0)).shape == (1, 0)


def test_tuning_file_roundtrip(tmp_path):
    """Autotuner choices written by one process are read back by another
    (host only): loading a file and saving it again gives the same entries;
    malformed lines are rejected."""
    src = tmp_path / "in.txt"
    src.write_text("# comment\n2 1024 4 1\n2 512 4 0\n3 128 8 4\n")
    ok.ok_tuning_load(str(src))
    out = tmp_path / "out.txt"
    ok.ok_tuning_save(str(out))
    lines = {l for l in out.read_text().splitlines() if not l.startswith("#")}
    assert {"2 1024 4 1", "2 512 4 0", "3 128 8 4"} <= lines
    bad = tmp_path / "bad.txt"
    bad.write_text("2 64 4 9\n")                     # shape 9 does not exist
    with pytest.raises(ok.OkError):
        ok.ok_tuning_load(str(bad))


def test_experiment_driver_imports():
    import paper_1603_04570_gb300.experiments as ex
    assert callable(ex.energy) and callable(ex.table1)
