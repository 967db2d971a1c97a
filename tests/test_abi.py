"""The C ABI library builds, loads without a GPU, and exports every entry point
that include/*.h declares.  No compute call is made here."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = {}
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(msz_\w+)\s*\(", text, flags=re.M):
            names[m.group(1)] = os.path.basename(h)
    return names


def test_headers_declare_entry_points():
    names = _declared()
    for n in ("msz_directions", "msz_correct", "msz_segment", "msz_compare", "msz_correct_host",
              "msz_workspace_size", "msz_status_str"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2601_01787_gb300 import _build
    path = _build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_sizes_without_gpu():
    from paper_2601_01787_gb300 import api
    lib = api.load()
    assert api.status_str(api.OK) == "MSZ_OK"
    assert api.status_str(api.STUCK) == "MSZ_STUCK"
    assert lib.msz_workspace_size(api.grid_of((4, 5, 6))) > 4 * 5 * 6 * 13
    assert lib.msz_workspace_size(api.Grid(4, 0, 1, 1, 1)) == 0       # bad ndim
    assert lib.msz_workspace_size(api.Grid(2, 0, 3, 3, 2)) == 0       # 2D with nz != 1
    assert lib.msz_workspace_size(api.Grid(3, 0, 2048, 2048, 1024)) == 0  # > 2^31 - 1 vertices
    g = api.grid_of((4, 5, 6))
    base = lib.msz_workspace_size(g)
    assert lib.msz_workspace_size_rule(g, 0) == lib.msz_workspace_size_rule(g, 1) == base
    assert lib.msz_workspace_size_rule(g, 2) >= base + 4 * 4 * 5 * 6  # one candidate record a vertex
    assert lib.msz_workspace_size_rule(g, 3) == 0                      # no such rule


def test_invalid_arguments_rejected_on_host():
    """Argument checks run before any CUDA call, so they work without a GPU."""
    from paper_2601_01787_gb300 import api
    lib = api.load()
    g = api.grid_of((3, 4, 5))
    cnt = ctypes.c_int64()
    fake = ctypes.c_void_p(256)
    st = lib.msz_correct(None, fake, ctypes.c_float(0.1), g, fake, None, None, 0, ctypes.byref(cnt), None, None,
                         fake, 1 << 30, None)
    assert st == api.ERR_INVALID_ARG
    st = lib.msz_correct(fake, fake, ctypes.c_float(-1.0), g, fake, None, None, 0, ctypes.byref(cnt), None, None,
                         fake, 1 << 30, None)
    assert st == api.ERR_INVALID_ARG
    st = lib.msz_correct(fake, fake, ctypes.c_float(0.1), g, fake, None, None, 0, ctypes.byref(cnt), None, None,
                         fake, 16, None)
    assert st == api.ERR_WORKSPACE
    bad_opt = api.Options(7, 0, 0, 0, None, None, 0)
    st = lib.msz_correct(fake, fake, ctypes.c_float(0.1), g, fake, None, None, 0, ctypes.byref(cnt),
                         ctypes.byref(bad_opt), None, fake, 1 << 30, None)
    assert st == api.ERR_INVALID_ARG
    bad_hook = api.Options(0, 3, 0, 0, None, None, 0)  # test_fault takes 0, 1 or 2
    st = lib.msz_correct(fake, fake, ctypes.c_float(0.1), g, fake, None, None, 0, ctypes.byref(cnt),
                         ctypes.byref(bad_hook), None, fake, 1 << 30, None)
    assert st == api.ERR_INVALID_ARG


def test_learned_arguments_rejected_on_host():
    """The learned entry points check channels, modes, pointers and alignment
    before any CUDA call."""
    from paper_2601_01787_gb300 import api, learned
    lib = learned.lib()
    g3 = api.grid_of((4, 5, 130))
    g2 = api.grid_of((5, 130))
    a = ctypes.c_void_p(1 << 20)      # 16-byte aligned, never dereferenced
    odd = ctypes.c_void_p((1 << 20) + 8)
    F = ctypes.c_float
    conv = lib.msz_learned_conv
    ok_args = dict(x=a, cin=32, cout=32, mode=learned.MODE_RELU, grid=g3, img=a, bias=a, ob=a, of=None, mask=None)

    def call(**kw):
        d = dict(ok_args, **kw)
        return conv(d["x"], d["cin"], d["cout"], d["mode"], d["grid"], d["img"], d["bias"], d["ob"], d["of"],
                    d["mask"], None, None, F(0.0), 0, None, a, None)

    assert call(cin=8) == api.ERR_INVALID_ARG                       # unsupported channels
    assert call(cout=16) == api.ERR_INVALID_ARG                     # ReLU layers have 32 outputs
    assert call(mode=7) == api.ERR_INVALID_ARG                      # unknown mode
    assert call(grid=g2) == api.ERR_INVALID_ARG                     # 3D only
    assert call(x=odd) == api.ERR_INVALID_ARG                       # TMA needs 16-byte alignment
    assert call(bias=None) == api.ERR_INVALID_ARG
    assert call(mode=learned.MODE_DGRAD) == api.ERR_INVALID_ARG     # no mask
    assert call(mode=learned.MODE_HEAD, cout=16) == api.ERR_INVALID_ARG  # neither r nor g0 requested
    assert call(mode=learned.MODE_RAW, ob=None) == api.ERR_INVALID_ARG   # no FP32 output
    w = lib.msz_learned_wgrad
    assert w(a, 16, a, 16, g3, 16, 16, a, a, a, 1 << 30, None) == api.ERR_INVALID_ARG  # 16 -> 16 is not a layer
    assert w(a, 32, a, 32, g3, 33, 32, a, a, a, 1 << 30, None) == api.ERR_INVALID_ARG  # more real than padded
    assert lib.msz_learned_wgrad_workspace_size(16, 16) == 0
    assert lib.msz_learned_wgrad_workspace_size(32, 32) >= 27 * 32 * 32 * 4  # a partial per block at least
    assert lib.msz_learned_weight_image(a, 0, 32, 32, 32, 0, a, None) == api.ERR_INVALID_ARG
    assert lib.msz_learned_weight_image(a, 32, 32, 32, 48, 0, a, None) == api.ERR_INVALID_ARG
    assert lib.msz_learned_features(a, a, F(1e-3), g2, a, a, a, None) == api.ERR_INVALID_ARG
    assert lib.msz_learned_adam(a, a, a, a, 10, F(1e-3), F(0.9), F(0.999), F(1e-8), 0, None) == api.ERR_INVALID_ARG
    # (cin / 16) slab pairs x 9 (dx, dz) strips x 2 K halves x 5 dy blocks x cout rows x 16 bytes
    assert int(lib.msz_learned_weight_image_size(32, 16)) == 2 * 9 * 2 * 5 * 16 * 16
    assert int(lib.msz_learned_weight_image_size(16, 32)) == 1 * 9 * 2 * 5 * 32 * 16
    assert int(lib.msz_learned_weight_image_size(24, 32)) == 0


def test_relaxed_arguments_rejected_on_host():
    from paper_2601_01787_gb300 import api
    lib = api.load()
    fake = ctypes.c_void_p(256)
    cnt = ctypes.c_int64()
    g2 = api.grid_of((8, 9))
    g3 = api.grid_of((4, 5, 6))
    assert lib.msz_relaxed_workspace_size(g2) == 0
    assert lib.msz_relaxed_workspace_size(g3) > lib.msz_workspace_size(g3)
    st = lib.msz_correct_relaxed(fake, fake, ctypes.c_float(0.1), g2, fake, None, None, 0, ctypes.byref(cnt), None,
                                 None, fake, 1 << 30, None)
    assert st == api.ERR_INVALID_ARG  # 3D only
    opt, _ = api._options("halve", 0, 0, None, 0, 0, 1)  # the test hook is not offered here
    st = lib.msz_correct_relaxed(fake, fake, ctypes.c_float(0.1), g3, fake, None, None, 0, ctypes.byref(cnt),
                                 ctypes.byref(opt), None, fake, 1 << 30, None)
    assert st == api.ERR_INVALID_ARG
    opt, _ = api._options("halve", 0, 0, None, 0, 0, 0, -1)  # negative local cap
    st = lib.msz_correct_relaxed(fake, fake, ctypes.c_float(0.1), g3, fake, None, None, 0, ctypes.byref(cnt),
                                 ctypes.byref(opt), None, fake, 1 << 30, None)
    assert st == api.ERR_INVALID_ARG
    st = lib.msz_correct_relaxed(fake, fake, ctypes.c_float(0.1), g3, fake, None, None, 0, ctypes.byref(cnt), None,
                                 None, fake, 16, None)
    assert st == api.ERR_WORKSPACE


def test_edit_encoding_sizes_and_arguments_on_host():
    from oracle import edits as E
    from paper_2601_01787_gb300 import api
    lib = api.load()
    for count in (0, 1, 3, 256, 257, 100000):
        nb = (count + 255) // 256
        table = 16 + 10 * nb + (-(10 * nb) % 4)
        assert lib.msz_edits_encoded_bound(count) == table + 8 * count
        assert lib.msz_edits_workspace_size(count) >= 256 + 10 * nb
    worst = E.encode([0, 1 << 30, (1 << 31) - 1], [0, 0, 0])  # 30-bit gaps, 32-bit distances
    assert len(worst) <= lib.msz_edits_encoded_bound(3)
    assert lib.msz_edits_encoded_bound(-1) == 0 and lib.msz_edits_workspace_size(-1) == 0
    fake = ctypes.c_void_p(256)
    nbytes = ctypes.c_size_t()
    cnt = ctypes.c_int64()
    ws = 1 << 20
    enc = lib.msz_edits_encode
    assert enc(None, fake, 10, fake, 3, fake, 64, ctypes.byref(nbytes), fake, ws, None) == api.ERR_INVALID_ARG
    assert enc(fake, fake, 10, fake, 11, fake, 64, ctypes.byref(nbytes), fake, ws, None) == api.ERR_INVALID_ARG
    assert enc(fake, fake, 10, None, 3, fake, 64, ctypes.byref(nbytes), fake, ws, None) == api.ERR_INVALID_ARG
    assert enc(fake, fake, 10, fake, 3, ctypes.c_void_p(258), 64, ctypes.byref(nbytes), fake, ws,
               None) == api.ERR_INVALID_ARG  # stream not 4-byte aligned
    assert enc(fake, fake, 10, fake, 3, fake, 64, ctypes.byref(nbytes), fake, 8, None) == api.ERR_WORKSPACE
    dec = lib.msz_edits_decode
    assert dec(None, 64, fake, 10, ctypes.byref(cnt), fake, ws, None) == api.ERR_INVALID_ARG
    assert dec(fake, 15, fake, 10, ctypes.byref(cnt), fake, ws, None) == api.ERR_INVALID_ARG
    assert dec(ctypes.c_void_p(257), 64, fake, 10, ctypes.byref(cnt), fake, ws, None) == api.ERR_INVALID_ARG


def test_pipeline_arguments_on_host():
    from paper_2601_01787_gb300 import api
    lib = api.load()
    g = api.grid_of((6, 7, 8))
    assert lib.msz_pipeline_workspace_size(g, 10) >= 2 * lib.msz_host_workspace_size(g, 10)
    assert lib.msz_pipeline_workspace_size(api.Grid(4, 0, 1, 1, 1), 10) == 0
    assert lib.msz_pipeline_workspace_size(g, -1) == 0
    h = ctypes.c_void_p()
    fake = ctypes.c_void_p(256)
    assert lib.msz_pipeline_create(g, 10, fake, 1 << 30, None) == api.ERR_INVALID_ARG
    assert lib.msz_pipeline_create(g, -1, fake, 1 << 30, ctypes.byref(h)) == api.ERR_INVALID_ARG
    assert lib.msz_pipeline_create(g, 10, fake, 64, ctypes.byref(h)) == api.ERR_WORKSPACE
    assert lib.msz_pipeline_create(g, 10, ctypes.c_void_p(260), 1 << 30, ctypes.byref(h)) == api.ERR_INVALID_ARG
    cnt = ctypes.c_int64()
    assert lib.msz_pipeline_submit(None, fake, fake, ctypes.c_float(0.1), fake, fake, fake, None) == api.ERR_INVALID_ARG
    assert lib.msz_pipeline_collect(None, ctypes.byref(cnt), None) == api.ERR_INVALID_ARG
    lib.msz_pipeline_destroy(None)  # a no-op


def test_encoded_pipeline_arguments_on_host():
    from paper_2601_01787_gb300 import api
    lib = api.load()
    g = api.grid_of((6, 7, 8))
    assert lib.msz_pipeline_workspace_size_encoded(g, 10) > lib.msz_pipeline_workspace_size(g, 10)
    assert lib.msz_pipeline_workspace_size_encoded(g, -1) == 0
    h = ctypes.c_void_p()
    fake = ctypes.c_void_p(256)
    assert lib.msz_pipeline_create_encoded(g, 10, fake, 64, ctypes.byref(h)) == api.ERR_WORKSPACE
    assert lib.msz_pipeline_create_encoded(g, 10, fake, 1 << 30, None) == api.ERR_INVALID_ARG
    cnt, nb = ctypes.c_int64(), ctypes.c_size_t()
    assert lib.msz_pipeline_submit_encoded(None, fake, fake, ctypes.c_float(0.1), fake, 64, None) == \
        api.ERR_INVALID_ARG
    assert lib.msz_pipeline_collect_encoded(None, ctypes.byref(cnt), ctypes.byref(nb), None) == api.ERR_INVALID_ARG


def test_batch_arguments_rejected_on_host():
    """msz_batch_workspace_size and the batch's argument and workspace checks
    run before any CUDA call."""
    from paper_2601_01787_gb300 import api
    lib = api.load()
    fake = 256

    def fields(shapes, **kw):
        arr = (api.Field * len(shapes))()
        for k, shp in enumerate(shapes):
            fk = arr[k]
            fk.d_f = fk.d_fhat = fk.d_out = fake
            fk.xi = kw.get("xi", 0.1)
            fk.grid = api.grid_of(shp)
            fk.edit_capacity = kw.get("cap", 0)
            if fk.edit_capacity > 0 and not kw.get("no_lists"):
                fk.d_edit_idx = fk.d_edit_delta = fake
        return arr

    good = fields([(4, 5, 6), (7, 3, 9)])
    size = lib.msz_batch_workspace_size(2, good, 0)
    assert size > 0
    assert lib.msz_batch_workspace_size(2, good, 8) < size             # a smaller sweep cap, a smaller log
    assert lib.msz_batch_workspace_size(0, good, 0) == 0
    assert lib.msz_batch_workspace_size(api.BATCH_MAX_FIELDS + 1, fields([(2, 2, 2)] * 257), 0) == 0
    assert lib.msz_batch_workspace_size(1, fields([(5, 6)]), 0) == 0       # 3D only
    assert lib.msz_batch_workspace_size(2, good, api.BATCH_MAX_SWEEPS + 1) == 0

    plan = ctypes.c_void_p()

    def create(arr, n=None, opt=None, ws_bytes=1 << 40):
        n = len(arr) if n is None else n
        return lib.msz_batch_plan_create(n, arr, ctypes.byref(opt) if opt is not None else None, fake, ws_bytes,
                                         None, ctypes.byref(plan))

    def options(**kw):
        opt, _ = api._options(kw.get("rule", "halve"), kw.get("max_sweeps", 0), kw.get("dense", 0), None, 0)
        opt.test_fault = kw.get("fault", 0)
        if kw.get("g_init"):
            opt.d_g_init = fake
        return opt

    assert create(good, n=0) == api.ERR_INVALID_ARG
    assert create(fields([(5, 6)])) == api.ERR_INVALID_ARG                       # 2D field
    assert create(good, opt=options(rule="below")) == api.ERR_INVALID_ARG  # HALVE or SNAP only
    assert create(good, opt=options(g_init=True)) == api.ERR_INVALID_ARG        # no proposed start
    assert create(good, opt=options(fault=1)) == api.ERR_INVALID_ARG            # no test hook
    assert create(good, opt=options(max_sweeps=api.BATCH_MAX_SWEEPS + 1)) == api.ERR_INVALID_ARG
    assert create(good, opt=options(dense=-2)) == api.ERR_INVALID_ARG
    assert create(fields([(4, 5, 6)], xi=-1.0)) == api.ERR_INVALID_ARG
    assert create(fields([(4, 5, 6)], xi=float("inf"))) == api.ERR_INVALID_ARG
    assert create(fields([(4, 5, 6)], cap=-1)) == api.ERR_INVALID_ARG
    assert create(fields([(4, 5, 6)], cap=10, no_lists=True)) == api.ERR_INVALID_ARG  # lists asked for, no buffers
    assert create(good, ws_bytes=size - 1) == api.ERR_WORKSPACE
    assert not plan.value  # no plan was made
