"""The device Philox4x32-10 of the sweep kernels (both forms: round keys bumped per
round, and precomputed) against CUDA's own Philox4x32-10 function (curand_kernel.h)
on 2^20 counter/key pairs: a pin of the device generator by a third implementation,
beside the published known-answer vectors that pin the oracle's."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1411_5512_gb300", "csrc")

SOURCE = r"""
#include <curand_kernel.h>
#include <cstdio>
#include <vector>
#include "ea_device.cuh"

__global__ void cmp_kernel(int n, uint4 *ours, uint4 *ours_rk, uint4 *ref)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const uint32_t u = (uint32_t)i;
    const uint4 c = make_uint4(u * 2654435761u, u ^ 0x5bd1e995u, u << 7, ~u);
    const uint32_t k0 = 0x12345678u + u * 0x9E3779B9u, k1 = 0xCAFEBABEu ^ (u * 0x85EBCA6Bu);
    ours[i] = ea::dev::philox10(c, k0, k1);
    uint32_t rk[20];
    for (int r = 0; r < 10; ++r) {
        rk[2 * r] = k0 + (uint32_t)r * 0x9E3779B9u;
        rk[2 * r + 1] = k1 + (uint32_t)r * 0xBB67AE85u;
    }
    ours_rk[i] = ea::dev::philox10_rk(c, rk);
    ref[i] = curand_Philox4x32_10(c, make_uint2(k0, k1));
}

int main()
{
    const int n = 1 << 20;
    uint4 *d = nullptr;
    if (cudaMalloc(&d, 3 * sizeof(uint4) * n) != cudaSuccess)
        return 2;
    cmp_kernel<<<(n + 255) / 256, 256>>>(n, d, d + n, d + 2 * n);
    std::vector<uint4> h(3 * (size_t)n);
    if (cudaMemcpy(h.data(), d, 3 * sizeof(uint4) * n, cudaMemcpyDeviceToHost) != cudaSuccess)
        return 3;
    cudaFree(d);
    long bad = 0;
    for (int i = 0; i < n; ++i) {
        const uint4 a = h[i], b = h[n + i], c = h[2 * (size_t)n + i];
        bad += (a.x != c.x || a.y != c.y || a.z != c.z || a.w != c.w);
        bad += (b.x != c.x || b.y != c.y || b.z != c.z || b.w != c.w);
    }
    std::printf("compared %d counters, mismatches %ld\n", n, bad);
    return bad == 0 ? 0 : 1;
}
"""


def _nvcc():
    path = shutil.which("nvcc")
    if path is None and os.path.exists("/usr/local/cuda/bin/nvcc"):
        path = "/usr/local/cuda/bin/nvcc"
    return path


def test_device_philox_matches_cuda_philox(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    cu = tmp_path / "philox_vs_cuda.cu"
    cu.write_text(SOURCE)
    exe = tmp_path / "philox_vs_cuda"
    r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17",
                        "-I" + CSRC, str(cu), "-o", str(exe)], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "mismatches 0" in r.stdout
