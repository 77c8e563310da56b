"""The C ABI library builds, loads without a GPU and exports every function
that include/*.h declares; host-side validation needs no device."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2405_14551_gb300 import build
    build.build()
    import paper_2405_14551_gb300.lbcg as L
    return L.load_library()


def declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(hdr).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(lb_[A-Za-z0-9_]+)\s*\(", txt, re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_core_calls():
    names = declared_functions()
    for core in ("lb_create", "lb_init_droplets", "lb_step", "lb_fields", "lb_destroy"):
        assert core in names


def test_every_declared_symbol_is_exported(lib):
    path = os.path.join(ROOT, "paper_2405_14551_gb300", "liblbcg.so")
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(lib, n)


def test_validation_without_gpu(lib):
    import paper_2405_14551_gb300.lbcg as L
    bad = [
        (L.make_grid(0, 4, 4), L.make_params()),
        (L.make_grid(4, 4, 4, walls=8), L.make_params()),
        (L.make_grid(4, 2, 4, walls=2), L.make_params()),
        (L.make_grid(4, 4, 4), L.make_params(tau_a=0.5)),
        (L.make_grid(4, 4, 4), L.make_params(beta=1.5)),
        (L.make_grid(4, 4, 4), L.make_params(A_h=0.1, h_max=9.0)),
        (L.make_grid(4, 4, 4), L.make_params(A_h=0.1, h_min=4.0, h_max=3.0)),
        (L.make_grid(4, 4, 4), L.make_params(g_mode=3)),
        (L.make_grid(4, 4, 4), L.make_params(storage=7)),
        (L.make_grid(4, 4, 4), L.make_params(storage="moment_f32")),  # moment storage needs collision = 1
        (L.make_grid(4, 4, 4), L.make_params(g=(float("nan"), 0.0, 0.0))),
        (L.make_grid(1 << 11, 1 << 11, 1 << 10), L.make_params()),
        (L.make_grid(4, 4, 4), L.make_params(model=2)),
        (L.make_grid(4, 4, 4), L.make_params(model=1, G=7.5, storage="reduced_f32")),  # Shan-Chen needs two sets
        (L.make_grid(4, 4, 4), L.make_params(model=1, G=7.5, A_h=0.1)),
        (L.make_grid(4, 4, 4), L.make_params(model=1, G=7.5, collision=1)),
        (L.make_grid(4, 4, 4), L.make_params(model=1, G=7.5, psi0=0.0)),
    ]
    for grid, params in bad:
        with pytest.raises(L.LBError) as ei:
            L.lb_create(grid, params)
        assert ei.value.code == L.LB_EINVAL
    # a valid request fails only for want of a device here
    try:
        import torch
        have = torch.cuda.is_available()
    except Exception:
        have = False
    if not have:
        with pytest.raises(L.LBError) as ei:
            L.lb_create(L.make_grid(8, 8, 8), L.make_params())
        assert ei.value.code == L.LB_ECUDA
    assert lib.lb_strerror(L.LB_EUNSTABLE).decode().startswith("unstable")
    assert L.lb_launch_count() >= 0


def test_null_handle_rejected(lib):
    import paper_2405_14551_gb300.lbcg as L
    assert lib.lb_step(None, 1) == L.LB_EINVAL
    assert lib.lb_check(None) == L.LB_EINVAL
    assert lib.lb_destroy(None) == L.LB_OK
    assert lib.lb_time(None) == -1
    assert lib.lb_set_tile(None, 0) == L.LB_EINVAL
    assert lib.lb_phi_monitor(None, None, None, None) == L.LB_EINVAL
    assert lib.lb_copy_state(None, None) == L.LB_EINVAL
    assert lib.lb_surrogate_load(None, b"x") == L.LB_EINVAL
    assert lib.lb_surrogate_predict(None, None) == L.LB_EINVAL
    assert lib.lb_get_tile(None) == -1


def test_conv_argument_checks_without_gpu(lib):
    """The convolution entry points validate their arguments on the host
    before any launch (null tensors, channel counts, extents)."""
    import paper_2405_14551_gb300.lbcg as L
    st = ctypes.c_void_p(16)
    assert lib.lbnn_conv3d_fwd(None, 16, None, 27, None, None, None, 16, 0, 8, 16, 4, 1, 0, 0, st, None) == L.LB_EINVAL
    buf = ctypes.c_void_p(256)  # never dereferenced: every call below is rejected first
    assert lib.lbnn_conv3d_fwd(buf, 24, buf, 27, None, buf, None, 16, 0, 8, 16, 4, 1, 0, 0, st, None) == L.LB_EINVAL
    assert lib.lbnn_conv3d_fwd_upcat(None, 32, buf, 64, buf, None, buf, None, 32, 0, 16, 16, 4, 1, 0, 1, st,
                                     None) == L.LB_EINVAL
    assert lib.lbnn_conv3d_fwd_upcat(buf, 24, buf, 64, buf, None, buf, None, 32, 0, 16, 16, 4, 1, 0, 1, st,
                                     None) == L.LB_EINVAL
    assert lib.lbnn_conv3d_fwd_upcat(buf, 32, buf, 64, buf, None, buf, None, 32, 0, 16, 8, 4, 1, 0, 1, st,
                                     None) == L.LB_EINVAL  # ny % 16
    assert lib.lbnn_conv3d_fwd_upcat(buf, 32, buf, 64, buf, None, buf, None, 32, 0, 16, 16, 3, 1, 0, 1, st,
                                     None) == L.LB_EINVAL  # odd nz


def test_conv_wait_limit_setting_without_gpu(lib):
    """The convolutions' wait limit is a process-wide host setting: it starts
    at the header's default, a set returns the previous value, and a null
    status word is rejected before any CUDA call."""
    import paper_2405_14551_gb300.lbcg as L
    with open(os.path.join(ROOT, "include", "lbnn.h")) as f:
        hdr = f.read()
    m = re.search(r"#define LBNN_WAIT_LIMIT_DEFAULT \(1u << (\d+)\)", hdr)
    assert m and L.LBNN_WAIT_LIMIT_DEFAULT == 1 << int(m.group(1))
    prev = L.lbnn_set_wait_limit(0)
    assert prev == L.LBNN_WAIT_LIMIT_DEFAULT
    assert L.lbnn_set_wait_limit(prev) == 0
    assert L.lbnn_set_wait_limit(prev) == prev
    assert lib.lbnn_check_status(None, None) == L.LB_EINVAL


def test_model_constants_agree_between_header_and_binding():
    import re

    import paper_2405_14551_gb300.lbcg as L
    h = open(os.path.join(ROOT, "include", "lbcg.h")).read()
    consts = dict(re.findall(r"#define (LB_MODEL_\w+) (\d+)", h))
    assert consts == {"LB_MODEL_COLOUR_GRADIENT": "0", "LB_MODEL_SHAN_CHEN": "1"}
    names = [f[0] for f in L.lb_params._fields_]
    assert names[-3:] == ["model", "G", "psi0"]


def test_storage_formats_agree_between_header_and_binding():
    """The binding's storage names, and the algorithmic bytes per node update
    it reports, follow the LB_STORAGE_* formats the header defines."""
    import paper_2405_14551_gb300.lbcg as L
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "lbcg.h")).read()
    defs = {m.group(1).lower(): int(m.group(2)) for m in re.finditer(r"#define LB_STORAGE_(\w+) (\d+)", hdr)}
    assert defs == L.STORAGE
    # one read + one write of the stored state per node update
    per_lattice = {"twoset_f32": 2 * 27 * 4, "reduced_f32": 27 * 4 + 16, "reduced_f16": 27 * 2 + 16,
                   "twoset_f64": 2 * 27 * 8, "moment_f32": 10 * 4 + 16}
    for name, st in L.STORAGE.items():
        assert L.BYTES_PER_NODE[st] == 2 * per_lattice[name], name


def test_tile_count_agrees_between_library_and_binding(lib):
    """The binding's tile count (which the bench's autotuner walks) is the
    library's: the tile table has that many shapes, each a whole number of
    warps, and lb_set_tile's documented range ends there."""
    import paper_2405_14551_gb300.lbcg as L
    csrc = os.path.join(ROOT, "paper_2405_14551_gb300", "csrc")
    with open(os.path.join(csrc, "internal.h")) as f:
        m = re.search(r"constexpr int NUM_TILES = (\d+);", f.read())
    assert m and int(m.group(1)) == L.NUM_TILES
    with open(os.path.join(csrc, "step_kernels.cu")) as f:
        m = re.search(r"kTiles\[NUM_TILES\] = \{(.*?)\};", f.read(), re.S)
    shapes = re.findall(r"\{(\d+), (\d+), (\d+)\}", m.group(1))
    assert len(shapes) == L.NUM_TILES
    assert all(int(x) * int(y) % 32 == 0 for x, y, _ in shapes)
    with open(os.path.join(ROOT, "include", "lbcg.h")) as f:
        assert f"(0..{L.NUM_TILES - 1}:" in f.read()
    assert lib.lb_set_tile(None, 0) == L.LB_EINVAL
