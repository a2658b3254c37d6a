// Allocation-free variant of the phase-field diagnostics reduction.
//
// Some callers cannot allocate device memory: code running inside a memory
// pool that forbids cudaMalloc, a host application whose allocator owns the
// whole device, or a real-time loop where an allocation would block.  For them
// pf_diagnostics_noalloc computes the same six FP64 reductions as
// pf_diagnostics directly from a phase field the caller already holds on the
// device, with no context and no allocation: the per-block partial sums live in
// one file-scope device array of fixed size, which the CUDA runtime reserves on
// each GPU by the time of the library's first call there (with lazy module
// loading, at that first call).
#include <cmath>

#include "../../include/dualpf.h"
#include "reduce.cuh"

namespace pf {

// Partial sums of up to kNoAllocBlocks reduction blocks (RED_N doubles each),
// followed by RED_N slots for the final sums: 1 MiB in total.
constexpr int kNoAllocBlocks = 16384;
constexpr int kNoAllocPerThread = 32;  // elements a thread folds per block pass
static __device__ __align__(256) double g_noalloc_scratch[(size_t)(kNoAllocBlocks + 1) * RED_N];

// Fixed-order sum of the block partials into the last RED_N slots.
__global__ void k_noalloc_final(double* __restrict__ scratch, int nblocks) {
  __shared__ double sh[RED_N][256];
  for (int q = 0; q < RED_N; ++q) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += scratch[(size_t)b * RED_N + q];
    sh[q][threadIdx.x] = s;
  }
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int q = 0; q < RED_N; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < RED_N; ++q) scratch[(size_t)kNoAllocBlocks * RED_N + q] = sh[q][0];
}

}  // namespace pf

extern "C" int pf_diagnostics_noalloc(const pf_grid_desc* g, const pf_params* prm, const void* phi_device,
                                      double out[6], void* stream) {
  using namespace pf;
  auto fail = [](int code, const char*) { return code; };
  if (!g || !prm || !phi_device || !out) return fail(PF_ERR_ARG, "null argument");
  if (g->nx < 2 || g->ny < 1 || g->nz < 2 || !(g->lx > 0)) return fail(PF_ERR_ARG, "bad grid");
  // PF_MIXED_Z64 and PF_MIXED_Z2F store phi as float, like PF_MIXED
  if (g->precision != PF_FP64 && g->precision != PF_MIXED && g->precision != PF_MIXED_Z64 &&
      g->precision != PF_MIXED_Z2F)
    return fail(PF_ERR_ARG, "bad precision");
  if (!(prm->eta > 0) || !(prm->sigma > 0)) return fail(PF_ERR_ARG, "eta and sigma must be > 0");
  Dims d{};
  d.nx = g->nx;
  d.ny = g->ny;
  d.nz = g->nz;
  d.dim = g->ny == 1 ? 2 : 3;
  d.r = g->dual ? 2 : 1;
  d.ry = d.dim == 3 ? d.r : 1;
  d.rs = d.r == 2 ? 1 : 0;
  d.rys = d.ry == 2 ? 1 : 0;
  d.fnx = d.r * g->nx;
  d.fny = d.ry * g->ny;
  d.fnz = d.r * g->nz;
  d.dx = g->lx / g->nx;
  d.h = d.dx / d.r;
  const size_t n = (size_t)d.fnx * d.fny * d.fnz;
  const size_t per_block = (size_t)256 * kNoAllocPerThread;
  const size_t nb = (n + per_block - 1) / per_block;
  if (nb > (size_t)kNoAllocBlocks)
    return fail(PF_ERR_UNSUPPORTED, "phase field larger than the fixed scratch allows (max 134217728 fine cells)");
  Phys p{};
  p.eta = prm->eta;
  p.lam = 3.0 * prm->sigma * prm->eta / (2.0 * std::sqrt(2.0));
  p.cos_bot = std::cos(prm->theta_bot_deg * M_PI / 180.0);
  p.cos_top = std::cos(prm->theta_top_deg * M_PI / 180.0);
  // Resolve the device address of the array on every call: it is cheap,
  // allocates nothing, and stays right after a cudaDeviceReset (which starts
  // a new context in which the array has a new address).
  double* scratch = nullptr;
  {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(PF_ERR_CUDA, cudaGetErrorString(e));
    }
    scratch = static_cast<double*>(ptr);
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const double dy = d.dim == 3 ? d.h : g->ly;
  if (g->precision == PF_FP64)
    k_reduce<double><<<(int)nb, 256, 0, st>>>(static_cast<const double*>(phi_device), d, p, prm->sigma, dy, scratch);
  else
    k_reduce<float><<<(int)nb, 256, 0, st>>>(static_cast<const float*>(phi_device), d, p, prm->sigma, dy, scratch);
  k_noalloc_final<<<1, 256, 0, st>>>(scratch, (int)nb);
  double s[RED_N];
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s, scratch + (size_t)kNoAllocBlocks * RED_N, sizeof(s), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(PF_ERR_CUDA, cudaGetErrorString(e));
  const double hd = std::pow(d.h, d.dim), hw = std::pow(d.h, d.dim - 1);
  out[0] = s[0] * hd;
  out[1] = p.lam * s[1] * hd + s[2] * hw;
  out[2] = s[3] * hw;
  out[3] = s[4] / s[7];
  out[4] = s[5] / s[7];
  out[5] = s[6] / s[7];
  return PF_OK;
}
