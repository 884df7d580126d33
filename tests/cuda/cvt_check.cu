// Checks the integer FP64 <-> FP32 conversions of the solve kernels
// (cvt_f32, cvt_f64 in fdpf_ops.cuh) against the hardware conversions
// (round to nearest even) on seeded values: normal doubles of many
// exponents, exact FP32 values, random FP32 bit patterns.  Prints the count
// of disagreements outside the documented cases (NaN input -> infinity;
// magnitudes below the FP32 normal range -> signed zero; exact ties, where
// cvt_f32 rounds away from zero) and exits non-zero on any.
#include <cstdio>
#include <cstring>
#include <cmath>
#include <cuda_runtime.h>
#include "../../paper_1803_03290_gb300/csrc/fdpf_ops.cuh"

using namespace gpcg;

__global__ void check(int n, const double* x, const float* y, unsigned* bad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double xv = x[i];
  const unsigned a = __float_as_uint(cvt_f32(xv)), b = __float_as_uint(__double2float_rn(xv));
  if (a != b) {
    const bool nan_in = xv != xv;
    const bool tiny = fabs(xv) < 1.1754943508222875e-38;
    // an exact tie: the 29 dropped bits are 1 followed by zeros
    const unsigned long long bits = (unsigned long long)__double_as_longlong(xv);
    const bool tie = (bits & 0x1fffffffull) == 0x10000000ull;
    if (!(nan_in && (a & 0x7fffffffu) == 0x7f800000u) && !tiny && !tie) atomicAdd(bad, 1u);
  }
  const float yv = y[i];
  const double c = cvt_f64(yv), d = (double)yv;
  const bool sub = fabsf(yv) < 1.17549435e-38f;
  if (!sub && __double_as_longlong(c) != __double_as_longlong(d)) {
    if (!(yv != yv && c != c)) atomicAdd(bad + 1, 1u);
  }
}

int main() {
  const int n = 1 << 22;
  double* hx = new double[n];
  float* hy = new float[n];
  unsigned long long s = 0x9E3779B97F4A7C15ull;
  for (int i = 0; i < n; ++i) {
    s ^= s << 13; s ^= s >> 7; s ^= s << 17;
    const unsigned long long r = s;
    double v;
    switch (i % 3) {
      case 0: v = std::ldexp(1.0 + (double)(r & ((1ull << 52) - 1)) / 4503599627370496.0,
                             (int)((r >> 52) % 240) - 120);
              if (r >> 63) v = -v;
              break;
      case 1: { unsigned u = (unsigned)(r >> 17); float f; std::memcpy(&f, &u, 4); v = f; break; }
      default: v = ((double)(r >> 11) / 9007199254740992.0 - 0.5) * 8.0; break;
    }
    hx[i] = v;
    unsigned u = (unsigned)(r >> 29);
    float f;
    std::memcpy(&f, &u, 4);
    hy[i] = f;
  }
  double* dx; float* dy; unsigned* bad;
  if (cudaMalloc(&dx, (size_t)n * 8) != cudaSuccess || cudaMalloc(&dy, (size_t)n * 4) != cudaSuccess ||
      cudaMalloc(&bad, 8) != cudaSuccess) { std::printf("alloc failed\n"); return 2; }
  cudaMemcpy(dx, hx, (size_t)n * 8, cudaMemcpyHostToDevice);
  cudaMemcpy(dy, hy, (size_t)n * 4, cudaMemcpyHostToDevice);
  cudaMemset(bad, 0, 8);
  check<<<(n + 255) / 256, 256>>>(n, dx, dy, bad);
  unsigned h[2] = {0, 0};
  const cudaError_t e = cudaMemcpy(h, bad, 8, cudaMemcpyDeviceToHost);
  std::printf("%s f64->f32 disagreements %u, f32->f64 disagreements %u, of %d values\n",
              cudaGetErrorString(e), h[0], h[1], n);
  cudaFree(dx); cudaFree(dy); cudaFree(bad);
  delete[] hx; delete[] hy;
  return (e != cudaSuccess || h[0] || h[1]) ? 1 : 0;
}
