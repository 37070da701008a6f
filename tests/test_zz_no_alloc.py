"""ad_filter_static: the filter G for callers that cannot let a library
allocate device memory (start-up-reserved real-time codes, memory owned by
another allocator, code that must not synchronize the device). Its scratch
is a fixed device array inside the library; this file checks, through the C
ABI, that two calls in a row give the same field as the allocating
ad_filter entry point and as the CPU oracle's filter (Eq. df2), within the
filter's parity tolerance, including the largest documented field (one
128^3 float32 field), and that a request above the array's size is refused.
It is named to run last so that a failure here never hides the rest of the
suite."""

import ctypes

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

TOL = {"f32": 3e-6, "f64": 1e-13}


def _lib(gad):
    lib = gad.load()
    lib.ad_filter_static.argtypes = [ctypes.POINTER(gad.ad_grid), ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_int, ctypes.c_void_p]
    lib.ad_filter_static.restype = ctypes.c_int
    return lib


def _grid(gad, shape, dtype, gamma):
    g = gad.ad_grid()
    g.ndim = len(shape)
    rev = list(reversed(shape)) + [1] * (3 - len(shape))
    for i in range(3):
        g.n[i] = int(rev[i])
    g.dtype = gad.AD_F32 if dtype == "f32" else gad.AD_F64
    g.gamma = float(gamma)
    return g


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("shape,batch,dtype,gamma", [((512, 512), 3, "f32", 0.01), ((2048, 2048), 1, "f32", 0.01),
                                                     ((48, 64, 96), 2, "f32", 0.1), ((128, 128, 128), 1, "f32", 0.1),
                                                     ((128, 128), 2, "f64", 0.1)])
def test_static_filter_matches_allocating_filter_and_oracle(gad, shape, batch, dtype, gamma):
    import torch
    lib = _lib(gad)
    tdt = torch.float32 if dtype == "f32" else torch.float64
    rng = np.random.default_rng(11)
    stream = torch.cuda.current_stream()
    g = _grid(gad, shape, dtype, gamma)
    for call in range(2):                      # two calls in a row share the scratch
        u = torch.tensor(rng.standard_normal((batch,) + shape), dtype=tdt, device="cuda")
        ref = gad.filter(u, gamma, ndim=len(shape))
        out = torch.full_like(u, float("nan"))
        st = lib.ad_filter_static(ctypes.byref(g), ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                  batch, ctypes.c_void_p(stream.cuda_stream))
        assert st == gad.AD_OK, (call, st)
        torch.cuda.synchronize()
        o, r = out.double().cpu().numpy(), ref.double().cpu().numpy()
        uin = u.double().cpu().numpy()
        for b in range(batch):
            assert _rel(o[b], r[b]) < TOL[dtype], (call, b, _rel(o[b], r[b]))
            # element by element against the oracle: relative L2 and the largest
            # pointwise deviation, both at the filter's tolerance
            ora = oracle.filter_field(uin[b], gamma)
            e2 = _rel(o[b], ora)
            einf = float(np.max(np.abs(o[b] - ora)) / np.max(np.abs(ora)))
            assert e2 < TOL[dtype] and einf < 10 * TOL[dtype], (call, b, e2, einf)


def test_static_filter_rejects_oversize_requests(gad):
    import torch
    lib = _lib(gad)
    # two 128^3 float32 fields need 2 x 17 MB of spectra: above the 32 MiB array
    v = torch.zeros((2, 128, 128, 128), device="cuda")
    g3 = _grid(gad, (128, 128, 128), "f32", 0.1)
    st = lib.ad_filter_static(ctypes.byref(g3), ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(v.data_ptr()), 2,
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == gad.AD_ERR_ARG
    u = torch.zeros((2, 2048, 2048), device="cuda")
    g = _grid(gad, (2048, 2048), "f32", 0.01)
    st = lib.ad_filter_static(ctypes.byref(g), ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(u.data_ptr()), 2,
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == gad.AD_ERR_ARG
    g = _grid(gad, (2048, 2048), "f32", 0.0)
    st = lib.ad_filter_static(ctypes.byref(g), ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(u.data_ptr()), 1,
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == gad.AD_ERR_ARG
