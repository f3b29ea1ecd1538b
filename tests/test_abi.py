"""The C-ABI library loads and exports every symbol include/heat.h declares (no GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**\s*(heat_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    b = __graft_entry__._build_module()
    b.build()
    return ctypes.CDLL(b.LIB)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["heat_create_mesh", "heat_sim_create", "heat_set_coeffs", "heat_step",
                     "heat_solve_transient", "heat_apply", "heat_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert missing == []


def test_binding_covers_the_header():
    import paper_1905_07622_gb300.api as api

    assert set(declared_functions()) <= set(api.EXPORTED)


def test_host_side_argument_checks_without_gpu(lib):
    import paper_1905_07622_gb300.api as api

    with pytest.raises(api.HeatError) as e:
        api.heat_create_mesh(0, 3, 3)
    assert e.value.status == api.HEAT_ERR_ARG
    with pytest.raises(api.HeatError):
        api.heat_create_mesh(2, 2, 2, extent=(1.0, -1.0, 1.0))
    for dims in [(2000, 2000, 2000), (2**31 - 1, 1, 1), (1290, 1290, 1290)]:  # >= 2^31 - 1 nodes
        with pytest.raises(api.HeatError) as e:
            api.heat_create_mesh(*dims)
        assert e.value.status == api.HEAT_ERR_ARG
    m = api.heat_create_mesh(3, 4, 5)
    assert api.heat_mesh_sizes(m) == (4 * 5 * 6, 60)
    api.heat_destroy_mesh(m)
    p = api.heat_params_default()
    assert p.resid_period == 50 and p.theta == 0.5


def test_server_create_fails_cleanly_without_a_device(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1905_07622_gb300.api as api

    with pytest.raises(api.HeatError) as e:
        api.heat_server_create(1 << 30, 4)
    assert e.value.status == api.HEAT_ERR_CUDA


def test_tuning_table_host_logic(lib):
    import paper_1905_07622_gb300.api as api

    n = api.heat_tuning_num_variants()
    assert n >= 2
    shapes = [api.heat_tuning_variant(v) for v in range(n)]
    assert all(s["seg_width"] in (16, 32) and s["rows"] >= 1 and s["warps"] >= 1 for s in shapes)
    with pytest.raises(api.HeatError):
        api.heat_tuning_variant(n)
    old = api.heat_tuning_get()
    assert old == {"variant": [-1, 0, 0], "seg_nodes": [512, 512, 512], "pw_quads": [2, 4, 4],
                   "open_w": [2, 2, 2], "loop": [0, 0, 0]}
    try:
        api.heat_tuning_set([-1, n - 1, 0], [256, 1024, 2048], [1, 2, 4], [1, 0, 1], [0, 1, 0])
        assert api.heat_tuning_get() == {"variant": [-1, n - 1, 0], "seg_nodes": [256, 1024, 2048],
                                         "pw_quads": [1, 2, 4], "open_w": [1, 0, 1], "loop": [0, 1, 0]}
        no64 = [v for v in range(n) if not shapes[v]["has_fp64"]]
        bad = [([-1, n, 0], [512] * 3), ([-2, 0, 0], [512] * 3), ([-1, 0, 0], [16, 512, 512]),
               ([-1, 0, 0], [512, 512, (1 << 20) + 1])]
        if no64:
            bad.append(([no64[0], 0, 0], [512] * 3))
        for variant, seg in bad:
            with pytest.raises(api.HeatError) as e:
                api.heat_tuning_set(variant, seg)
            assert e.value.status == api.HEAT_ERR_ARG
        for quads in ([3, 4, 4], [2, 0, 4], [2, 4, 8]):
            with pytest.raises(api.HeatError):
                api.heat_tuning_set([-1, 0, 0], [512] * 3, quads)
        for ow in ([3, 1, 1], [0, -1, 1]):
            with pytest.raises(api.HeatError):
                api.heat_tuning_set([-1, 0, 0], [512] * 3, [2, 4, 4], ow)
        # the persistent iteration is 0 or 1, and only for the FP32 paths
        for lp in ([1, 0, 0], [0, 2, 0], [0, 0, -1]):
            with pytest.raises(api.HeatError) as e:
                api.heat_tuning_set([-1, 0, 0], [512] * 3, [2, 4, 4], [2, 2, 2], lp)
            assert e.value.status == api.HEAT_ERR_ARG
        # a rejected table leaves the last good one in place
        assert api.heat_tuning_get() == {"variant": [-1, n - 1, 0], "seg_nodes": [256, 1024, 2048],
                                         "pw_quads": [1, 2, 4], "open_w": [1, 0, 1], "loop": [0, 1, 0]}
    finally:
        api.heat_tuning_set(old["variant"], old["seg_nodes"], old["pw_quads"], old["open_w"], old["loop"])


def test_grid_barrier_probe_checks_its_arguments(lib):
    import paper_1905_07622_gb300.api as api

    for bps, reps in ((0, 10), (17, 10), (1, 0), (1, 100001)):
        with pytest.raises(api.HeatError) as e:
            api.heat_probe_grid_barrier(bps, reps)
        assert e.value.status == api.HEAT_ERR_ARG


def test_loop_wait_hook_checks_its_arguments(lib):
    import paper_1905_07622_gb300.api as api

    for extra, limit in ((2, 0.0), (0, -1.0), (1, 61.0), (0, float("nan"))):
        with pytest.raises(api.HeatError) as e:
            api.heat_debug_loop_wait(extra, limit)
        assert e.value.status == api.HEAT_ERR_ARG
    api.heat_debug_loop_wait(0, 0.0)  # the defaults


@pytest.mark.parametrize("bad", ["f32_coef", "short_coef", "short_x", "long_y", "empty_dot", "cpu"])
def test_noalloc_binding_rejects_bad_tensors_before_the_call(bad):
    """heat_apply_dot_noalloc's binding checks dtype, length and device of every
    buffer: the C entry point cannot, and a short device buffer would be read
    or written out of bounds."""
    torch = pytest.importorskip("torch")
    import paper_1905_07622_gb300.api as api
    nx, ny, nz = 3, 4, 5
    nn = (nx + 1) * (ny + 1) * (nz + 1)
    f64 = dict(dtype=torch.float64)
    t = {"coef": torch.zeros(2 * nx * ny * nz, **f64), "x": torch.zeros(nn, **f64),
         "y": torch.zeros(nn, **f64), "xdoty": torch.zeros(1, **f64)}
    if bad == "f32_coef":
        t["coef"] = t["coef"].float()
    elif bad == "short_coef":
        t["coef"] = t["coef"][:-1]
    elif bad == "short_x":
        t["x"] = t["x"][:-2]
    elif bad == "long_y":
        t["y"] = torch.zeros(nn + 1, **f64)
    elif bad == "empty_dot":
        t["xdoty"] = torch.zeros(0, **f64)
    with pytest.raises((ValueError, TypeError)):
        api.heat_apply_dot_noalloc(nx, ny, nz, (1.0, 1.0, 1.0), 1e-3, 0.5, 0, t["coef"], t["x"], t["y"], t["xdoty"])
