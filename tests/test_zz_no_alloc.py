"""The allocation-free lower-bound entry point (messi_lower_bounds_noalloc).

It exists for callers that may not allocate device memory while they run:
an embedding that owns a fixed device-memory budget, or a latency-critical
loop that must not stall in cudaMalloc / cudaFree.  Its scratch is one fixed
array inside the library, shared by every call.  This file is collected last
so that, if it fails, a run that stops at the first failure has already run
every other test; it passes both alone in a fresh process and after the
other tests.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _lib_call(m, name, ix, q, dist, window, out, stream):
    return getattr(m._lib, name)(ix.handle, ctypes.c_void_p(q.data_ptr()), dist, window,
                                 ctypes.c_void_p(out.data_ptr()), stream)


def test_noalloc_lower_bounds_match_allocating_entry_point():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import paper_2110_07519_gb300 as m

    x = synth.random_walks(50_000, 256, seed=4242)
    ix = m.messi_build(torch.from_numpy(x).cuda(), 16, 256)
    qs = synth.query_mix(x, 2, seed=4243)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # the first call on a device looks up the scratch array (and may load the
    # library's device code), so the memory check below starts after it
    warm = torch.empty(x.shape[0], dtype=torch.float32, device="cuda")
    q0 = torch.from_numpy(qs[0]).cuda()
    assert _lib_call(m, "messi_lower_bounds_noalloc", ix, q0, 0, 0, warm, stream) == 0, m.messi_last_error()
    torch.cuda.synchronize()
    # two calls in a row, the second on the array the first left behind
    for call, (dist, window) in enumerate([(m.MESSI_ED, 0), (m.MESSI_DTW, 25)]):
        q = torch.from_numpy(qs[call]).cuda()
        ref = torch.empty(x.shape[0], dtype=torch.float32, device="cuda")
        out = torch.full((x.shape[0],), -1.0, dtype=torch.float32, device="cuda")
        assert _lib_call(m, "messi_lower_bounds", ix, q, dist, window, ref, stream) == 0, m.messi_last_error()
        torch.cuda.synchronize()
        # the call itself allocates nothing: free device memory is unchanged
        free0 = torch.cuda.mem_get_info()[0]
        assert _lib_call(m, "messi_lower_bounds_noalloc", ix, q, dist, window, out, stream) == 0, \
            m.messi_last_error()
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        m.messi_check(ix)
        a, b = ref.cpu().numpy(), out.cpu().numpy()
        assert np.allclose(b, a, rtol=1e-5, atol=0.0)
        assert np.array_equal(b, a)          # same kernels, same arithmetic
        assert (b >= 0).all()


def test_noalloc_non_finite_query_leaves_output_and_reports():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import paper_2110_07519_gb300 as m

    x = synth.random_walks(5000, 256, seed=4244)
    ix = m.messi_build(torch.from_numpy(x).cuda(), 16, 256)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    q = torch.from_numpy(x[3].copy()).cuda()
    q[17] = float("nan")
    out = torch.full((x.shape[0],), -7.0, dtype=torch.float32, device="cuda")
    assert _lib_call(m, "messi_lower_bounds_noalloc", ix, q, 0, 0, out, stream) == 0
    torch.cuda.synchronize()
    with pytest.raises(m.MessiError) as e:
        m.messi_check(ix)
    assert e.value.status == 1
    assert (out.cpu().numpy() == -7.0).all()      # left unwritten
    # a finite query afterwards works on the same scratch
    q[17] = 0.0
    ref = m.messi_lower_bounds(ix, q)
    assert _lib_call(m, "messi_lower_bounds_noalloc", ix, q, 0, 0, out, stream) == 0
    torch.cuda.synchronize()
    m.messi_check(ix)
    assert np.array_equal(out.cpu().numpy(), ref.cpu().numpy())


def test_noalloc_rejects_what_it_cannot_do_without_allocating():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import paper_2110_07519_gb300 as m

    lib = m._lib
    stream = ctypes.c_void_p(0)
    x = synth.random_walks(1000, 256, seed=1)
    ix = m.messi_build(torch.from_numpy(x).cuda(), 16, 256)
    q = np.ascontiguousarray(x[0])
    out_host = np.empty(1000, np.float32)
    # host buffers would need staging memory
    assert lib.messi_lower_bounds_noalloc(ix.handle, ctypes.c_void_p(q.ctypes.data), 0, 0,
                                          ctypes.c_void_p(out_host.ctypes.data), stream) == 1
    # longer series than the fixed scratch holds
    y = synth.random_walks(300, 4096, seed=2)
    iy = m.messi_build(torch.from_numpy(y).cuda(), 16, 256)
    qd = torch.from_numpy(y[0]).cuda()
    od = torch.empty(300, dtype=torch.float32, device="cuda")
    st = lib.messi_lower_bounds_noalloc(iy.handle, ctypes.c_void_p(qd.data_ptr()), 0, 0,
                                        ctypes.c_void_p(od.data_ptr()), stream)
    assert st == 1 and "2048" in m.messi_last_error()
