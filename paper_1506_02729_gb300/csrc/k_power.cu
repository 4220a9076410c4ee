// k_power.cu - scalars, gridding and bin reduction of the power-spectrum
// path (Sec. III.A of the paper):
//   scalars (alpha, I_22, I_33, N_0, S_3; eqs. I22def, N0true, Noise0),
//   gridding of galaxies and randoms (eq. mapFFT, CIC/TSC) with L^ab (eq. Lab),
//   the fixed-order FP64 reduction of the z-pass's per-block bin sums.
// The three FFT passes are in k_fftpass.cu.
#include <cuda_runtime.h>
#include <stdint.h>

#include "fkp_internal.h"

namespace fkp {

// ----------------------------------------------------------------------------
// helpers
// ----------------------------------------------------------------------------

struct KahanF {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) {
    float y = v - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// Block-wide FP64 sum of one value per thread; the result is valid in thread 0.
__device__ double block_sum_f64(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int i = 0; i < nw; ++i) r += sh[i];
  }
  return r;
}

__device__ __forceinline__ float fkp_weight(const CatDev& c, long long i, float Pfkp) {
  return c.w ? __ldg(c.w + i) : 1.0f / (1.0f + __ldg(c.nbar + i) * Pfkp);
}

__device__ __forceinline__ float pw(const float* h, int e) {
  // h = {1, x, x^2, x^3, x^4}
  return e == 0 ? 1.f : (e == 1 ? h[1] : (e == 2 ? h[2] : (e == 3 ? h[3] : h[4])));
}

// ----------------------------------------------------------------------------
// a1: FP64 scalars.  Per-thread compensated FP32 sums, per-block FP64 sums.
// ----------------------------------------------------------------------------

__global__ void __launch_bounds__(256) k_scalars(CatDev c, int is_ran, float Pfkp, double* __restrict__ part) {
  __shared__ double sh[32];
  KahanF s_w, s_w2, s_w3, s_nw2, s_n2w3;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < c.n;
       i += (long long)gridDim.x * blockDim.x) {
    const float w = fkp_weight(c, i, Pfkp);
    const float w2 = w * w;
    s_w.add(w);
    s_w2.add(w2);
    s_w3.add(w2 * w);
    if (is_ran) {
      const float nb = __ldg(c.nbar + i);
      s_nw2.add(nb * w2);
      s_n2w3.add(nb * nb * w2 * w);
    }
  }
  double* out = part + (size_t)blockIdx.x * SC_NSUM;
  double v;
  if (!is_ran) {
    v = block_sum_f64(s_w.value(), sh);  if (threadIdx.x == 0) out[SC_G_W] = v;
    v = block_sum_f64(s_w2.value(), sh); if (threadIdx.x == 0) out[SC_G_W2] = v;
    v = block_sum_f64(s_w3.value(), sh); if (threadIdx.x == 0) out[SC_G_W3] = v;
  } else {
    v = block_sum_f64(s_w.value(), sh);    if (threadIdx.x == 0) out[SC_R_W] = v;
    v = block_sum_f64(s_w2.value(), sh);   if (threadIdx.x == 0) out[SC_R_W2] = v;
    v = block_sum_f64(s_w3.value(), sh);   if (threadIdx.x == 0) out[SC_R_W3] = v;
    v = block_sum_f64(s_nw2.value(), sh);  if (threadIdx.x == 0) out[SC_R_NW2] = v;
    v = block_sum_f64(s_n2w3.value(), sh); if (threadIdx.x == 0) out[SC_R_N2W3] = v;
  }
}

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

// ----------------------------------------------------------------------------
// a2: gridding.  Every tap is rounded once to a 2^-40 fixed-point integer and
// added with a 64-bit integer atomic, so the grid does not depend on the
// order in which objects are processed (deterministic, batch invariant).
// ----------------------------------------------------------------------------

template <int P>
__device__ __forceinline__ void taps(float u, int& i0, float* wt) {
  if (P == 2) {
    const float f = floorf(u);
    const float d = u - f;
    i0 = (int)f;
    wt[0] = 1.f - d;
    wt[1] = d;
  } else {
    const float f = floorf(u + 0.5f);
    const float d = u - f;
    i0 = (int)f - 1;
    const float a = 0.5f - d, b = 0.5f + d;
    wt[0] = 0.5f * a * a;
    wt[1] = 0.75f - d * d;
    wt[2] = 0.5f * b * b;
  }
}

template <int P>
__global__ void __launch_bounds__(256) k_assign(CatDev c, int is_ran, GeomDev g, float obx, float oby, float obz,
                                                const double* __restrict__ ds, unsigned long long* __restrict__ grid,
                                                unsigned long long* __restrict__ gridw, int* __restrict__ err,
                                                double* __restrict__ labpart) {
  __shared__ double sh[32];
  const float alpha = (float)ds[DS_ALPHA];
  const int N = g.N;
  KahanF lab[LAB_NSUM];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < c.n;
       i += (long long)gridDim.x * blockDim.x) {
    const float w = fkp_weight(c, i, g.P_fkp);
    const float px = __ldg(c.x + i), py = __ldg(c.y + i), pz = __ldg(c.z + i);
    const float v = is_ran ? -alpha * w : w;
    const float vw = is_ran ? alpha * alpha * w * w : w * w;
    const float ux = (px - g.ox) * g.invH, uy = (py - g.oy) * g.invH, uz = (pz - g.oz) * g.invH;
    int ix, iy, iz;
    float wx[P], wy[P], wz[P];
    taps<P>(ux, ix, wx);
    taps<P>(uy, iy, wy);
    taps<P>(uz, iz, wz);
    const bool finite = (ux >= 0.f) && (ux < (float)N) && (uy >= 0.f) && (uy < (float)N) && (uz >= 0.f) &&
                        (uz < (float)N);
    if (!g.periodic) {
      const bool inside = finite && ix >= 1 && iy >= 1 && iz >= 1 && ix + P - 1 <= N - 2 && iy + P - 1 <= N - 2 &&
                          iz + P - 1 <= N - 2;
      if (!inside) {
        atomicOr(err, 1);
        continue;
      }
    } else if (!(fabsf(ux) < 1e8f && fabsf(uy) < 1e8f && fabsf(uz) < 1e8f)) {
      atomicOr(err, 2);
      continue;
    }
#pragma unroll
    for (int a = 0; a < P; ++a) {
      int zz = iz + a;
      zz = zz < 0 ? zz + N * ((-zz + N - 1) / N) : zz;
      zz %= N;
#pragma unroll
      for (int b = 0; b < P; ++b) {
        int yy = iy + b;
        yy = yy < 0 ? yy + N * ((-yy + N - 1) / N) : yy;
        yy %= N;
        const float wzy = wz[a] * wy[b];
        const size_t row = ((size_t)zz * N + yy) * N;
#pragma unroll
        for (int cc = 0; cc < P; ++cc) {
          int xx = ix + cc;
          xx = xx < 0 ? xx + N * ((-xx + N - 1) / N) : xx;
          xx %= N;
          const float t = wzy * wx[cc];
          atomicAdd(grid + row + xx, (unsigned long long)__float2ll_rn(v * t * kFixScaleF));
          if (gridw) atomicAdd(gridw + row + xx, (unsigned long long)__float2ll_rn(vw * t * kFixScaleF));
        }
      }
    }
    if (is_ran && labpart) {
      float hx, hy, hz;
      if (g.los_inf) {
        hx = g.lx; hy = g.ly; hz = g.lz;
      } else {
        const float dx = px - obx, dy = py - oby, dz = pz - obz;
        const float r2 = dx * dx + dy * dy + dz * dz;
        const float inv = r2 > 0.f ? rsqrtf(r2) : 0.f;
        hx = dx * inv; hy = dy * inv; hz = dz * inv;
      }
      lab[0].add(w * hx * hx);
      lab[1].add(w * hy * hy);
      lab[2].add(w * hz * hz);
      lab[3].add(w * hx * hy);
      lab[4].add(w * hy * hz);
      lab[5].add(w * hz * hx);
    }
  }
  if (is_ran && labpart) {
#pragma unroll
    for (int q = 0; q < LAB_NSUM; ++q) {
      const double v = block_sum_f64(lab[q].value(), sh);
      if (threadIdx.x == 0) labpart[(size_t)blockIdx.x * LAB_NSUM + q] = v;
    }
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
__global__ void __launch_bounds__(256) k_reduce_bins(const double* __restrict__ part, const int* __restrict__ partc,
                                                     int nblk, int nbins, double* __restrict__ out,
                                                     long long* __restrict__ outc) {
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

// ----------------------------------------------------------------------------
// host-side launch wrappers (called by the C ABI)
// ----------------------------------------------------------------------------

cudaError_t launch_scalars(const CatDev& c, int is_ran, float Pfkp, double* part, int nblk, cudaStream_t s) {
  if (c.n > 0) k_scalars<<<nblk, 256, 0, s>>>(c, is_ran, Pfkp, part);
  else cudaMemsetAsync(part, 0, sizeof(double) * SC_NSUM * nblk, s);
  return cudaGetLastError();
}

cudaError_t launch_scalars_finalize(const double* part, int nbg, int nbr, long long ng, long long nr, int amode,
                                    double* ds, cudaStream_t s) {
  k_scalars_finalize<<<1, 32, 0, s>>>(part, nbg, nbr, ng, nr, amode, ds);
  return cudaGetLastError();
}

cudaError_t launch_assign(const CatDev& c, int is_ran, const GeomDev& g, const double obs[3], const double* ds,
                          unsigned long long* grid, unsigned long long* gridw, int* err, double* labpart, int nblk,
                          cudaStream_t s) {
  if (c.n == 0) {
    if (labpart) cudaMemsetAsync(labpart, 0, sizeof(double) * LAB_NSUM * nblk, s);
    return cudaGetLastError();
  }
  if (g.assign == 2)
    k_assign<2><<<nblk, 256, 0, s>>>(c, is_ran, g, (float)obs[0], (float)obs[1], (float)obs[2], ds, grid, gridw, err,
                                     labpart);
  else
    k_assign<3><<<nblk, 256, 0, s>>>(c, is_ran, g, (float)obs[0], (float)obs[1], (float)obs[2], ds, grid, gridw, err,
                                     labpart);
  return cudaGetLastError();
}

cudaError_t launch_lab_finalize(const double* labpart, int nblk, double* out, cudaStream_t s) {
  k_lab_finalize<<<1, 32, 0, s>>>(labpart, nblk, out);
  return cudaGetLastError();
}

cudaError_t launch_reduce_bins(const double* part, const int* partc, int nblk, int nbins, double* out, long long* outc,
                               cudaStream_t s) {
  k_reduce_bins<<<(BQ_N + 1) * nbins, 256, 0, s>>>(part, partc, nblk, nbins, out, outc);
  return cudaGetLastError();
}

}  // namespace fkp
