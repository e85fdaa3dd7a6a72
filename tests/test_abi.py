"""The C-ABI library loads, exports every function include/tr.h declares, and
rejects bad arguments before touching the GPU.  No compute calls here."""

import ctypes
import os

import pytest

from paper_2506_09594_gb300 import tr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(tr.LIB_PATH):
        from paper_2506_09594_gb300 import build
        build.build()
    return tr.load()


def test_every_declared_function_is_exported(lib):
    names = tr.header_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
        assert name in tr._SIGS, "binding lacks " + name


def test_library_leaves_no_internal_symbol_undefined(lib):
    # a shared library links with undefined symbols and binds functions
    # lazily, so a helper declared in one translation unit and defined in none
    # would load here and fail only at its first call; every undefined symbol
    # must come from the C or C++ runtime (versioned) or be weak
    import shutil
    import subprocess
    if shutil.which("nm") is None:
        pytest.skip("nm not installed")
    out = subprocess.run(["nm", "-u", "-D", tr.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    bad = [ln.split()[-1] for ln in out.splitlines()
           if ln.split() and ln.split()[0] != "w" and "@" not in ln.split()[-1]]
    assert not bad, bad


def test_binding_struct_sizes_match_header_layout():
    # tr_params: 5 ints/enums, 12 doubles, 1 uint64, 1 pointer, with C padding
    assert ctypes.sizeof(tr.tr_problem) == 4 + 4 + 8 * 8 + 4 + 4 + 8 + 8
    assert ctypes.alignment(tr.tr_params) == 8
    assert ctypes.sizeof(tr.tr_step_info) % 8 == 0


def test_default_params(lib):
    p = tr.default_params()
    assert p.phi == tr.TR_PEN_MCP and p.psi == tr.TR_PEN_MCP
    assert p.mu0 == 1e-3 and p.mu_max == 1e10 and p.growth == 1.1 and p.tol == 1e-4
    assert p.engine == tr.TR_LR_RSVD and p.rank == 10 and p.oversample == 10
    assert p.power_iters == 1 and p.prec == tr.TR_PREC_FP32


def _init(lib, order, dims, dtype=tr.TR_F32, observed=1, mask=1, **kw):
    prob = tr.tr_problem()
    prob.order = order
    for i, d in enumerate(dims[:8]):
        prob.dims[i] = d
    prob.dtype = dtype
    prob.observed = observed
    prob.mask = mask
    prm = tr.default_params(**kw)
    h = ctypes.c_void_p()
    st = lib.tr_init(ctypes.byref(h), ctypes.byref(prob), ctypes.byref(prm), None)
    return st, h


def test_init_rejects_bad_arguments_without_a_gpu(lib):
    assert _init(lib, 1, [4])[0] == tr.TR_EINVAL                    # order < 2
    assert _init(lib, 9, [2] * 9)[0] == tr.TR_EINVAL                # order > 8
    assert _init(lib, 3, [4, 0, 3])[0] == tr.TR_EINVAL              # empty mode
    assert _init(lib, 3, [4, 4, 3], dtype=7)[0] == tr.TR_EINVAL     # dtype
    assert _init(lib, 3, [4, 4, 3], observed=None)[0] == tr.TR_EINVAL
    assert _init(lib, 3, [4, 4, 3], mu0=0.0)[0] == tr.TR_EINVAL
    assert _init(lib, 3, [4, 4, 3], power_iters=-1)[0] == tr.TR_EINVAL
    st, _ = _init(lib, 3, [4, 4, 100])                               # mode > 64
    assert st == tr.TR_EUNSUPPORTED
    msg = lib.tr_last_error(None).decode()
    assert "64" in msg
    assert lib.tr_free(None) == tr.TR_OK
    assert lib.tr_prox_step(None, None) == tr.TR_EINVAL


def test_library_refuses_missing_build(tmp_path):
    saved = tr._lib
    try:
        tr._lib = None
        with pytest.raises(RuntimeError):
            tr.load(str(tmp_path / "nope.so"))
    finally:
        tr._lib = saved


def test_tensor_core_precisions_need_fp32(lib):
    st, _ = _init(lib, 3, [8, 8, 4], dtype=tr.TR_F64, prec=tr.TR_PREC_BF16)
    assert st == tr.TR_EUNSUPPORTED
    st, _ = _init(lib, 3, [8, 8, 4], prec=tr.TR_PREC_TF32)
    assert st == tr.TR_EUNSUPPORTED


def test_model_file_roundtrip(tmp_path):
    import numpy as np
    w = np.random.default_rng(0).standard_normal(tr.TR_MLP_PARAMS).astype(np.float32)
    path = tmp_path / "m.bin"
    tr.save_model(str(path), w)
    raw = path.read_bytes()
    assert raw[:8] == b"TRRANK01" and len(raw) == 32 + 4 * tr.TR_MLP_PARAMS
    assert np.array_equal(tr.load_model(str(path)), w)
    with pytest.raises(ValueError):
        tr.save_model(str(path), w[:-1])


def test_mlp_param_count_export():
    from oracle import learned
    assert tr.load().tr_mlp_param_count() == tr.TR_MLP_PARAMS == learned.param_count()


def test_batch_and_graph_calls_validate_without_gpu(lib):
    b = ctypes.c_void_p()
    assert lib.tr_batch_create(ctypes.byref(b), 0, None, None, 0, None) == tr.TR_EINVAL
    assert b"bad arguments" in lib.tr_batch_last_error()
    assert lib.tr_batch_step(None, None) == tr.TR_EINVAL
    assert lib.tr_batch_free(None) == tr.TR_OK
    assert lib.tr_graph_mode(None, 1) == tr.TR_EINVAL
    assert lib.tr_set_tube_tile(None, 8) == tr.TR_EINVAL
    assert lib.tr_autotune(None, 1, None, None) == tr.TR_EINVAL
    assert lib.tr_set_slice_groups(None, 2) == tr.TR_EINVAL


def test_init_rejects_oversized_problems_without_a_gpu(lib):
    # slice panels beyond shared memory, sketches beyond the widest width,
    # adaptive blocks out of range, an engine that is not built, too many
    # slices: all refused before any device allocation
    st, _ = _init(lib, 3, [2048, 64, 4])                              # slice rows > 1024
    assert st == tr.TR_EUNSUPPORTED and "exceed" in lib.tr_last_error(None).decode()
    st, _ = _init(lib, 3, [512, 512, 4], rank=120, oversample=10)     # l = 130 > 96
    assert st == tr.TR_EUNSUPPORTED
    st, _ = _init(lib, 3, [64, 64, 4], engine=tr.TR_LR_ADAPTIVE, adapt_block=0)
    assert st == tr.TR_EINVAL
    st, _ = _init(lib, 3, [64, 64, 4], engine=tr.TR_LR_FULLSVD)
    assert st == tr.TR_EUNSUPPORTED
    st, _ = _init(lib, 3, [64, 64, 70000])                           # slices > 65535
    assert st == tr.TR_EUNSUPPORTED
    assert lib.tr_set_observed(None, None, None) == tr.TR_EINVAL
    assert lib.tr_read_residuals(None, None) == tr.TR_EINVAL
    assert lib.tr_slice_prox_tucker(None, None, None, 0.0, 1, 1, 1, 1, 0, 0, None, None, None,
                                    None) == tr.TR_EINVAL
    # shared-Tucker engine: (q + 1) l above 32 (l = 20, q = 1) or a mode size
    st, _ = _init(lib, 3, [64, 64, 4], engine=tr.TR_LR_TUCKER, rank=10, oversample=10)
    assert st == tr.TR_EUNSUPPORTED and "Tucker" in lib.tr_last_error(None).decode()
    st, _ = _init(lib, 3, [64, 10, 4], engine=tr.TR_LR_TUCKER, rank=4, oversample=2,
                  power_iters=1)
    assert st == tr.TR_EUNSUPPORTED


def test_handleless_error_messages_are_per_thread(lib):
    # a failed tr_init in one host thread does not overwrite the message
    # another thread reads for its own failed call
    import threading
    st, _ = _init(lib, 3, [4, 4, 100])                                # mode > 64
    assert st == tr.TR_EUNSUPPORTED
    mine = lib.tr_last_error(None).decode()
    seen = {}

    def other():
        s, _ = _init(lib, 3, [2048, 64, 4])                           # slice rows > 1024
        seen["st"] = s
        seen["msg"] = lib.tr_last_error(None).decode()

    t = threading.Thread(target=other)
    t.start()
    t.join()
    assert seen["st"] == tr.TR_EUNSUPPORTED and "exceed" in seen["msg"]
    assert lib.tr_last_error(None).decode() == mine and "64" in mine


def test_binding_keeps_the_current_and_previous_buffers_alive():
    # tr_set_observed switches buffer pairs while a step enqueued on the
    # previous pair may still run: the binding holds both, for plain handles
    # and for the borrowed handles of a batch (whose references the batch keeps)
    h = tr.Handle.__new__(tr.Handle)
    h._keep = ("M0", "m0")
    h._remember(("M1", "m1"))
    h._remember(("M2", "m2"))
    assert h._keep == ("M2", "m2") and h._keep_prev == ("M1", "m1")
    b = tr.Batch.__new__(tr.Batch)
    b._keep = [("A", "a"), ("B", "b")]
    b._keep_prev = [None, None]
    bh = tr.BorrowedHandle(None, (4, 4, 2), None, None, 0, owner=b, index=1)
    bh._remember(("C", "c"))
    del bh
    assert b._keep == [("A", "a"), ("C", "c")] and b._keep_prev == [None, ("B", "b")]
    assert not hasattr(tr.Batch, "set_observed")


def test_binding_refuses_bad_tensors_before_the_c_call(lib):
    # the C ABI sees only pointers: dtype, device, layout and size are checked
    # by the binding, with an error that is both a TrError (TR_EINVAL) and a
    # ValueError
    torch = pytest.importorskip("torch")
    need = tr._need
    x = torch.zeros((4, 6), dtype=torch.float32)
    need(x, "x", torch.float32, 24, device="cpu")
    need(None, "x", torch.float32, 24, device="cpu", optional=True)
    for args, what in (((x, "x", torch.float64, 24), "float64"),
                       ((x, "x", torch.float32, 25), "needs 25"),
                       ((x.t(), "x", torch.float32, 24), "contiguous"),
                       ((None, "x", torch.float32, 1), "required"),
                       ((x.numpy(), "x", torch.float32, 1), "torch tensor")):
        with pytest.raises(tr.TrArgError) as ei:
            need(*args, device="cpu")
        assert what in str(ei.value) and ei.value.status == tr.TR_EINVAL
        assert isinstance(ei.value, ValueError)
    with pytest.raises(tr.TrArgError, match="cuda"):
        need(x, "x", torch.float32, 24)
    # entry points refuse host tensors, wrong dtypes and short buffers
    M = torch.zeros((2, 4, 4))
    mask = torch.ones((2, 4, 4), dtype=torch.uint8)
    with pytest.raises(tr.TrArgError):
        tr.Handle(M, mask, (4, 4, 2))
    with pytest.raises(tr.TrArgError):
        tr.Handle(M.to(torch.int32), mask, (4, 4, 2))
    with pytest.raises(tr.TrArgError):
        tr.slice_prox_noalloc(M, M, 4, 1, 0.1, 0)
    with pytest.raises(tr.TrArgError):
        tr.mlp_forward(torch.zeros(tr.TR_MLP_PARAMS), torch.zeros((3, tr.TR_MLP_FEATURES)))
    with pytest.raises(tr.TrArgError):
        tr.Batch([(M, mask, (4, 4, 2))], tr.default_params())


def test_gradient_building_blocks_validate_without_gpu(lib):
    # tr_grad / tr_gradient_solve refuse bad arguments before any CUDA call
    dims = (ctypes.c_int64 * 3)(8, 6, 4)
    buf = ctypes.create_string_buffer(128)
    a, b = ctypes.c_void_p(256), ctypes.c_void_p(512)
    assert lib.tr_grad(7, 3, dims, 1, 0, a, b, None, buf, 128) == tr.TR_EINVAL
    assert lib.tr_grad(tr.TR_F32, 1, dims, 1, 0, a, b, None, buf, 128) == tr.TR_EINVAL
    assert lib.tr_grad(tr.TR_F32, 3, dims, 4, 0, a, b, None, buf, 128) == tr.TR_EINVAL
    assert lib.tr_grad(tr.TR_F32, 3, dims, 0, 0, a, b, None, buf, 128) == tr.TR_EINVAL
    assert lib.tr_grad(tr.TR_F32, 3, dims, 1, 0, a, a, None, buf, 128) == tr.TR_EINVAL
    assert b"distinct" in buf.value
    assert lib.tr_gradient_solve(tr.TR_F32, 3, dims, 0b1000, a, b, None, buf, 128) == tr.TR_EINVAL
    assert lib.tr_gradient_solve(tr.TR_F64, 3, dims, 0b011, a, a, None, buf, 128) == tr.TR_EINVAL
    zero = (ctypes.c_int64 * 3)(8, 0, 4)
    assert lib.tr_gradient_solve(tr.TR_F32, 3, zero, 0b011, a, b, None, buf, 128) == tr.TR_EINVAL
    big = (ctypes.c_int64 * 3)(4096, 6, 4)                  # a solved mode above 2048
    assert lib.tr_gradient_solve(tr.TR_F32, 3, big, 0b001, a, b, None, buf, 128) == \
        tr.TR_EUNSUPPORTED
    tall = (ctypes.c_int64 * 2)(1 << 23, 1)                 # mode-2 product rows beyond one grid
    assert lib.tr_gradient_solve(tr.TR_F32, 2, tall, 0b010, a, b, None, buf, 128) == \
        tr.TR_EUNSUPPORTED
    with pytest.raises(tr.TrArgError):
        tr.gradient_solve(pytest.importorskip("torch").zeros((4, 8, 6)), (8, 6, 4), (5,))


def test_onebit_create_validates_without_gpu(lib):
    dims = (ctypes.c_int64 * 3)(8, 6, 4)
    buf = ctypes.create_string_buffer(128)
    p = tr.onebit_params()
    a, b = ctypes.c_void_p(256), ctypes.c_void_p(512)
    ob = ctypes.c_void_p()

    def create(dt=tr.TR_F32, order=3, d=dims, m=10, idx=a, sgn=b, prm=p):
        return lib.tr_onebit_create(ctypes.byref(ob), dt, order, d, m, idx, sgn,
                                    ctypes.byref(prm), None, buf, 128)

    assert create(idx=None) == tr.TR_EINVAL
    assert create(m=0) == tr.TR_EINVAL
    assert create(dt=5) == tr.TR_EINVAL
    assert create(order=2) == tr.TR_EINVAL
    assert create(prm=tr.onebit_params(modes=0)) == tr.TR_EINVAL
    assert create(prm=tr.onebit_params(modes=[4])) == tr.TR_EINVAL
    assert create(prm=tr.onebit_params(mu0=0.0)) == tr.TR_EINVAL
    assert create(prm=tr.onebit_params(alpha=-1.0)) == tr.TR_EINVAL
    assert create(d=(ctypes.c_int64 * 3)(8, 0, 4)) == tr.TR_EINVAL
    assert create(d=(ctypes.c_int64 * 3)(1 << 16, 1 << 16, 4)) == tr.TR_EUNSUPPORTED
    assert b"entries" in buf.value
    assert lib.tr_onebit_step(None, None) == tr.TR_EINVAL
    assert lib.tr_onebit_free(None) == tr.TR_OK


def test_ctv_create_validates_without_gpu(lib):
    buf = ctypes.create_string_buffer(128)
    c = ctypes.c_void_p()

    def create(order=3, dims=(8, 6, 4), dtype=tr.TR_F32, obs=256, mask=512, **kw):
        pb = tr.tr_problem()
        pb.order = order
        for i, d in enumerate(dims):
            pb.dims[i] = d
        pb.dtype = dtype
        pb.observed = obs
        pb.mask = mask
        prm = tr.ctv_params(**kw)
        return lib.tr_ctv_create(ctypes.byref(c), ctypes.byref(pb), ctypes.byref(prm), None, buf,
                                 128)

    assert create(order=2, dims=(8, 6)) == tr.TR_EINVAL
    assert create(dtype=9) == tr.TR_EINVAL
    assert create(obs=None) == tr.TR_EINVAL
    assert create(modes=0) == tr.TR_EINVAL
    assert create(modes=[4]) == tr.TR_EINVAL
    assert create(mu0=-1.0) == tr.TR_EINVAL
    assert create(noise=7) == tr.TR_EINVAL
    assert create(dims=(8, 0, 4)) == tr.TR_EINVAL
    assert lib.tr_ctv_step(None, None) == tr.TR_EINVAL
    assert lib.tr_ctv_free(None) == tr.TR_OK


def test_model_bindings_refuse_bad_tensors(lib):
    torch = pytest.importorskip("torch")
    M = torch.zeros((4, 8, 6))
    mask = torch.ones((4, 8, 6), dtype=torch.uint8)
    with pytest.raises(tr.TrArgError):                 # host tensors
        tr.Ctv(M, mask, (8, 6, 4))
    with pytest.raises(tr.TrArgError):                 # integer observations
        tr.Ctv(M.to(torch.int32), mask, (8, 6, 4))
    idx = torch.zeros(10, dtype=torch.int64)
    sgn = torch.ones(10, dtype=torch.int8)
    with pytest.raises(tr.TrArgError):                 # host samples
        tr.OneBit((8, 6, 4), idx, sgn)
    with pytest.raises(tr.TrArgError):                 # signs as float
        tr.OneBit((8, 6, 4), idx, sgn.float())
    with pytest.raises(tr.TrArgError):
        tr.OneBit((8, 6, 4), idx, sgn, dtype=torch.float16)
    with pytest.raises(KeyError):
        tr.ctv_params(no_such_field=1)
    assert tr.onebit_params(modes=[2, 3]).modes == 0b110


def test_binding_structs_match_the_c_layout(tmp_path):
    # every field offset of the ABI structs, as the C compiler lays them out,
    # equals the ctypes binding's
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [("tr_problem", tr.tr_problem, {}), ("tr_params", tr.tr_params, {"lambda_": "lambda"}),
               ("tr_step_info", tr.tr_step_info, {}),
               ("tr_onebit_params", tr.tr_onebit_params, {"lambda_": "lambda"}),
               ("tr_ctv_params", tr.tr_ctv_params, {"lambda_": "lambda"})]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "tr.h"', "int main(void) {"]
    for cname, cls, rename in structs:
        lines.append('  printf("%s %%zu\\n", sizeof(%s));' % (cname, cname))
        for fname, _ in cls._fields_:
            c = rename.get(fname, fname)
            lines.append('  printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (cname, fname, cname, c))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(line.split() for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                      text=True).stdout.splitlines())
    for cname, cls, _ in structs:
        assert int(out[cname]) == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert int(out["%s.%s" % (cname, fname)]) == getattr(cls, fname).offset, (cname, fname)


def test_ad_tucker_prox_validates_without_gpu(lib):
    buf = ctypes.create_string_buffer(128)
    a, b = ctypes.c_void_p(256), ctypes.c_void_p(512)

    def call(dt=tr.TR_F32, n=4, n1=8, n2=6, A=a, G=b, tau=0.1, phi=tr.TR_PEN_L1, eps=1e-3, bs=4,
             dr=1e-12, mr=0, t=0):
        return lib.tr_slice_prox_ad_tucker(dt, n, n1, n2, A, G, tau, phi, 1.0, 4.0, eps, bs, dr,
                                           mr, 0, t, None, None, buf, 128)

    assert call(dt=3) == tr.TR_EINVAL
    assert call(n=0) == tr.TR_EINVAL
    assert call(bs=0) == tr.TR_EINVAL and call(bs=33) == tr.TR_EINVAL
    assert call(eps=0.0) == tr.TR_EINVAL
    assert call(G=a) == tr.TR_EINVAL
    assert call(phi=9) == tr.TR_EINVAL
    assert call(mr=-1) == tr.TR_EINVAL
    assert call(n=70000) == tr.TR_EUNSUPPORTED
