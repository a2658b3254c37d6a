// FP64 global reductions of the phase field (mass, free energy, wetted
// length, centroid).  Per-block partial sums are written in a fixed order and
// summed on the host, so results are deterministic.
#pragma once
#include "common.cuh"

namespace pf {

constexpr int RED_N = 8;  // sum phi, bulk energy density, wall energy, wetted, wx, wy, wz, w

// Rows of the fine mesh are taken in fixed groups of RGROUP consecutive rows,
// one group per block iteration; each thread position sums its elements of a
// group in the field's type and adds that to FP64 accumulators.  The group
// sums do not depend on the grid size, so any number of blocks gives the same
// FP32 partials (FP64 fields are accumulated in FP64 throughout).
constexpr int RGROUP = 8;

// The accumulators are Wide<T>: FP64, or Dual when derivatives are carried.
// The mass, the sum the method conserves, is accumulated in Wide<T> element by
// element, and with compensated FP32 storage (lo: the remainders of phi, or
// null) takes value + remainder: it is the exact sum of the stored field, so
// a drift it shows is the field's own, not the summation's.
template <class T>
__global__ void __launch_bounds__(256) k_reduce(const T* __restrict__ phi, Dims d, Phys p, double sigma, double dy,
                                                Wide<T>* __restrict__ partial, const T* __restrict__ lo = nullptr) {
  using W = Wide<T>;
  __shared__ W sh[RED_N][256];
  W acc[RED_N];
#pragma unroll
  for (int q = 0; q < RED_N; ++q) acc[q] = 0.0;
  W mass = 0.0;
  const int rows = d.fny * d.fnz, fnx = d.fnx;
  const size_t plane = (size_t)fnx * d.fny;
  const T h = (T)d.h, ih = (T)(1.0 / d.h), ie2 = (T)(1.0 / (p.eta * p.eta)), dyT = (T)dy;
  const T scb = (T)(sigma * p.cos_bot), sct = (T)(sigma * p.cos_top);
  const int ngroups = (rows + RGROUP - 1) / RGROUP;
  for (int grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
    T ga[RED_N];
#pragma unroll
    for (int q = 0; q < RED_N; ++q) ga[q] = (T)0;
    const int r1 = min(rows, (grp + 1) * RGROUP);
    for (int r = grp * RGROUP; r < r1; ++r) {
      const int k = r / d.fny, j = r - k * d.fny;
      const T* row = phi + (size_t)r * fnx;
      const T* rym = phi + ((size_t)k * d.fny + (j == 0 ? d.fny - 1 : j - 1)) * fnx;
      const bool wall = k == 0 || k == d.fnz - 1;
      const T* rw = k == 0 ? row + plane : row - plane;  // the second layer from the wall
      const T yj = ((T)j + (T)0.5) * dyT, zk = ((T)k + (T)0.5) * h;
      for (int i = threadIdx.x; i < fnx; i += blockDim.x) {
        const T c = row[i];
        mass += (W)c;
        if (lo) mass += (W)lo[(size_t)r * fnx + i];
        const T gx = (c - row[i == 0 ? fnx - 1 : i - 1]) * ih;
        T e = (T)0.5 * gx * gx;
        if (d.dim == 3) {
          const T gy = (c - rym[i]) * ih;
          e += (T)0.5 * gy * gy;
        }
        if (k > 0) {
          const T gz = (c - row[(ptrdiff_t)i - (ptrdiff_t)plane]) * ih;
          e += (T)0.5 * gz * gz;
        }
        e += (c * c - (T)1) * (c * c - (T)1) * (T)0.25 * ie2;
        ga[1] += e;
        if (wall && d.fnz > 1) {
          const T pw = (T)1.5 * c - (T)0.5 * rw[i];
          ga[2] += (k == 0 ? scb : sct) * pw * (pw * pw - (T)3) * (T)0.25;
          if (k == 0) ga[3] += (T)0.5 * ((T)1 + pw);
        }
        const T wgt = (T)0.5 * ((T)1 + c);
        ga[4] += wgt * ((T)i + (T)0.5) * h;
        ga[5] += wgt * yj;
        ga[6] += wgt * zk;
        ga[7] += wgt;
      }
    }
#pragma unroll
    for (int q = 1; q < RED_N; ++q) acc[q] += (W)ga[q];
  }
  acc[0] = mass;
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

// Sum of phi only (the finiteness check after steps): FP32 fields are read as
// float4 where the row length allows, each vector summed in FP32 and added in
// FP64; a NaN or Inf anywhere makes the sum non-finite.
template <class T>
__global__ void __launch_bounds__(256) k_sum_phi(const T* __restrict__ phi, size_t n, double* __restrict__ partial) {
  __shared__ double sh[256];
  double acc = 0.0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t i0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if constexpr (sizeof(T) == 4) {
    if (n % 4 == 0) {
      const float4* v = reinterpret_cast<const float4*>(phi);
      for (size_t i = i0; i < n / 4; i += stride) {
        const float4 a = v[i];
        acc += (double)((a.x + a.y) + (a.z + a.w));
      }
      i0 = n;  // done
    }
  }
  for (size_t i = i0; i < n; i += stride) acc += (double)phi[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

}  // namespace pf
