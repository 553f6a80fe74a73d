"""The integer-pipe FP64 helpers of the local solves (csrc/fp64_int.cuh) against the FP64
division and square root of the same GPU: reciprocal and square root within 1 ulp over
the exponent range and at the edges of the mantissa ranges the Newton iterations work on,
and exact integer constants.  A probe kernel is compiled from the header for this test."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

from paper_1606_03135_gb300 import build as B
from paper_1606_03135_gb300 import nodesets as NS

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PROBE = r'''
#include "fp64_int.cuh"
__global__ void k_probe(const double* x, double* s, double* r, const int* v, double* e, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        s[i] = rbffd::sqrt_fast(x[i]);
        r[i] = rbffd::rcp_fixed(x[i]);
        e[i] = rbffd::exact_double(v[i]);
    }
}
extern "C" int probe(const double* x, double* s, double* r, const int* v, double* e, int n) {
    k_probe<<<256, 256>>>(x, s, r, v, e, n);
    return (int)cudaDeviceSynchronize();
}
'''


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    d = tmp_path_factory.mktemp("probe")
    src = d / "probe.cu"
    src.write_text(PROBE)
    lib = d / "libprobe.so"
    subprocess.check_call([B.nvcc(), *B.ARCH, "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
                           "-shared", "-I", B.CSRC, str(src), "-o", str(lib)])
    L = C.CDLL(str(lib))
    L.probe.argtypes = [C.c_void_p] * 5 + [C.c_int]
    return L


def ulp_diff(a, b):
    ia = a.view(np.int64)
    ib = b.view(np.int64)
    return np.abs(ia - ib)


def test_sqrt_and_reciprocal_within_one_ulp_and_exact_integers(probe):
    u = NS.uniform(17, 400000)
    mant = 1.0 + u[:200000]
    expo = np.floor(NS.uniform(18, 200000) * 2040 - 1020).astype(np.int64)
    xs = [np.ldexp(mant, expo),                         # all exponents
          np.ldexp(1.0, np.arange(-1022, 1023)),          # powers of two (and of four)
          np.nextafter(np.ldexp(1.0, np.arange(-1020, 1020)), np.inf),
          np.nextafter(np.ldexp(1.0, np.arange(-1020, 1020)), 0.0),  # just below: m' near 4
          4.0 * u[200000:300000] ** 2,                     # the squared distances of the solves
          np.array([1.0, 2.0, 3.0, 4.0, 0.25, 1e-300, 1e300, 2.0 ** -1022])]
    x = np.concatenate(xs)
    x = x[np.isfinite(x) & (x > 0)]
    v = np.concatenate([np.arange(0, 5000), (NS.splitmix64(3, 5000) >> np.uint64(33)).astype(np.int64)])
    v = v.astype(np.int32)
    xd = torch.from_numpy(x).cuda()
    vd = torch.from_numpy(np.resize(v, x.size)).cuda()
    s = torch.empty_like(xd)
    r = torch.empty_like(xd)
    e = torch.empty_like(xd)
    assert probe.probe(xd.data_ptr(), s.data_ptr(), r.data_ptr(), vd.data_ptr(),
                       e.data_ptr(), x.size) == 0
    s_ref = torch.sqrt(xd).cpu().numpy()
    r_ref = (1.0 / xd).cpu().numpy()
    s, r, e = s.cpu().numpy(), r.cpu().numpy(), e.cpu().numpy()
    assert ulp_diff(s, s_ref).max() <= 1
    assert ulp_diff(r, r_ref).max() <= 1
    assert np.mean(s == s_ref) > 0.95 and np.mean(r == r_ref) > 0.95
    assert np.array_equal(e, np.resize(v, x.size).astype(np.float64))
