// k_power.cu - scalar finalize and bin reduction of the power-spectrum
// path (Sec. III.A of the paper):
//   the FP64 finalize of the scalars (alpha, I_22, I_33, N_0, S_3; eqs.
//   I22def, N0true, Noise0) and of L^ab (eq. Lab), and the fixed-order FP64
//   reduction of the z-pass's per-block bin sums.  Gridding is in
//   k_assign.cu, the three FFT passes in k_xpass.cu, k_ypass.cu and
//   k_zpass.cu.
#include <cuda_runtime.h>
#include <stdint.h>

#include "fkp_internal.h"

namespace fkp {

// ----------------------------------------------------------------------------
// helpers
// ----------------------------------------------------------------------------

// One block of 32 threads: fixed-order sums over the per-block partials and
// the derived scalars, all FP64.  Galaxy blocks are [0, nbg), random blocks
// [nbg, nbg + nbr).
__global__ void k_scalars_finalize(const double* __restrict__ part, int nbg, int nbr, long long ng, long long nr,
                                   int alpha_mode, double* __restrict__ ds) {
  __shared__ double tot[SC_NSUM];
  const int q = threadIdx.x;
  if (q < SC_NSUM) {
    const bool gal = q <= SC_G_W3;
    const int b0 = gal ? 0 : nbg, b1 = gal ? nbg : nbg + nbr;
    double s = 0.0;
    for (int b = b0; b < b1; ++b) s += part[(size_t)b * SC_NSUM + q];
    tot[q] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double Wg = tot[SC_G_W], Wr = tot[SC_R_W];
    const double a = alpha_mode == 0 ? Wg / Wr : (double)ng / (double)nr;
    ds[DS_ALPHA] = a;
    ds[DS_I22] = a * tot[SC_R_NW2];
    ds[DS_I33] = a * tot[SC_R_N2W3];
    ds[DS_N0] = tot[SC_G_W2] + a * a * tot[SC_R_W2];
    ds[DS_N0FKP] = a * (1.0 + a) * tot[SC_R_W2];
    ds[DS_S3] = tot[SC_G_W3] - a * a * a * tot[SC_R_W3];
    ds[DS_WG] = Wg;
    ds[DS_WR] = Wr;
    ds[DS_NG] = (double)ng;
    ds[DS_NR] = (double)nr;
  }
}

__global__ void k_lab_finalize(const double* __restrict__ labpart, int nblk, double* __restrict__ out) {
  const int q = threadIdx.x;
  if (q < LAB_NSUM) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += labpart[(size_t)b * LAB_NSUM + q];
    out[q] = s;
  }
}

// One block per (quantity, bin): fixed-order FP64 tree sum over the blocks.
// blockIdx.y picks the mock of a fused launch (partials at pstride / pcstride,
// bins contiguous per mock).
__global__ void __launch_bounds__(256) k_reduce_bins(const double* __restrict__ part, const int* __restrict__ partc,
                                                     int nblk, int nbins, double* __restrict__ out,
                                                     long long* __restrict__ outc, long long pstride,
                                                     long long pcstride) {
  part += (long long)blockIdx.y * pstride;
  partc += (long long)blockIdx.y * pcstride;
  out += (long long)blockIdx.y * BQ_N * nbins;
  outc += (long long)blockIdx.y * nbins;
  __shared__ double sh[32];
  const int row = blockIdx.x;  // 0 .. BQ_N*nbins (float rows) then nbins (count rows)
  double s = 0.0;
  if (row < BQ_N * nbins) {
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += part[(size_t)row * nblk + b];
    s = block_sum_f64(s, sh);
    if (threadIdx.x == 0) out[row] = s;
  } else {
    const int r = row - BQ_N * nbins;
    long long cs = 0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) cs += partc[(size_t)r * nblk + b];
    s = block_sum_f64((double)cs, sh);
    if (threadIdx.x == 0) outc[r] = (long long)s;
  }
}

// Diagnostic of the bounded wait: one block initialises an mbarrier that
// nothing ever arrives at and no copy targets, then waits on its first phase
// with the passes' bounded wait (mbar_wait_n) for `polls` polls.  flag gets
// 1 when the wait gave up (the expected outcome), 2 if it completed.
__global__ void k_wait_selftest(unsigned polls, int* __restrict__ flag) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && mbar_wait_n(&bar, 0u, flag, 1, polls)) atomicOr(flag, 2);
}

// ----------------------------------------------------------------------------
// host-side launch wrappers (called by the C ABI)
// ----------------------------------------------------------------------------

cudaError_t launch_scalars_finalize(const double* part, int nbg, int nbr, long long ng, long long nr, int amode,
                                    double* ds, cudaStream_t s) {
  k_scalars_finalize<<<1, 32, 0, s>>>(part, nbg, nbr, ng, nr, amode, ds);
  return cudaGetLastError();
}

cudaError_t launch_wait_selftest(unsigned polls, int* flag, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(polls, flag);
  return cudaGetLastError();
}

cudaError_t launch_lab_finalize(const double* labpart, int nblk, double* out, cudaStream_t s) {
  k_lab_finalize<<<1, 32, 0, s>>>(labpart, nblk, out);
  return cudaGetLastError();
}

cudaError_t launch_reduce_bins(const double* part, const int* partc, int nblk, int nbins, double* out, long long* outc,
                               cudaStream_t s, int nmock, long long pstride, long long pcstride) {
  k_reduce_bins<<<dim3((BQ_N + 1) * nbins, nmock), 256, 0, s>>>(part, partc, nblk, nbins, out, outc, pstride,
                                                                pcstride);
  return cudaGetLastError();
}

}  // namespace fkp
