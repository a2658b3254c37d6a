// FP64 global reductions of the phase field (mass, free energy, wetted
// length, centroid).  Per-block partial sums are written in a fixed order and
// summed on the host, so results are deterministic.
#pragma once
#include "common.cuh"

namespace pf {

constexpr int RED_N = 8;  // sum phi, bulk energy density, wall energy, wetted, wx, wy, wz, w

template <class T>
__global__ void k_reduce(const T* __restrict__ phi, Dims d, Phys p, double sigma, double dy, double* __restrict__ partial) {
  __shared__ double sh[RED_N][256];
  double acc[RED_N];
#pragma unroll
  for (int q = 0; q < RED_N; ++q) acc[q] = 0.0;
  const size_t n = (size_t)d.fnx * d.fny * d.fnz;
  const double h = d.h, ih = 1.0 / d.h, ie2 = 1.0 / (p.eta * p.eta);
  for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < n; id += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(id % d.fnx);
    const int j = (int)((id / d.fnx) % d.fny);
    const int k = (int)(id / ((size_t)d.fnx * d.fny));
    const double c = (double)phi[id];
    acc[0] += c;
    double gx = (c - (double)phi[fidx(d, wrap(i - 1, d.fnx), j, k)]) * ih;
    double e = 0.5 * gx * gx;
    if (d.dim == 3) {
      const double gy = (c - (double)phi[fidx(d, i, wrap(j - 1, d.fny), k)]) * ih;
      e += 0.5 * gy * gy;
    }
    if (k > 0) {
      const double gz = (c - (double)phi[fidx(d, i, j, k - 1)]) * ih;
      e += 0.5 * gz * gz;
    }
    e += (c * c - 1.0) * (c * c - 1.0) * 0.25 * ie2;
    acc[1] += e;
    if (k == 0 || k == d.fnz - 1) {
      const int k1 = (k == 0) ? 1 : d.fnz - 2;
      const double pw = 1.5 * c - 0.5 * (double)phi[fidx(d, i, j, k1)];
      const double cth = (k == 0) ? p.cos_bot : p.cos_top;
      double fw = sigma * cth * pw * (pw * pw - 3.0) * 0.25;
      acc[2] += fw;
      if (k == 0) acc[3] += 0.5 * (1.0 + pw);
    }
    const double wgt = 0.5 * (1.0 + c);
    acc[4] += wgt * (i + 0.5) * h;
    acc[5] += wgt * (j + 0.5) * dy;
    acc[6] += wgt * (k + 0.5) * h;
    acc[7] += wgt;
  }
#pragma unroll
  for (int q = 0; q < RED_N; ++q) sh[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
#pragma unroll
      for (int q = 0; q < RED_N; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0)
#pragma unroll
    for (int q = 0; q < RED_N; ++q) partial[(size_t)blockIdx.x * RED_N + q] = sh[q][0];
}

}  // namespace pf
