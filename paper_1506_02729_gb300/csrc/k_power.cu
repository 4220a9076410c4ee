// k_power.cu - the power-spectrum hot path (Sec. III.A of the paper):
//   scalars (alpha, I_22, I_33, N_0, S_3; eqs. I22def, N0true, Noise0),
//   gridding of galaxies and randoms (eq. mapFFT, CIC/TSC) with L^ab (eq. Lab),
//   x-pass: moment fields F x^_a x^_b (...) about the observer built per node
//           (eqs. Qij, Qijkl, Qab) and transformed along x (real-to-complex),
//   y-pass: transform along y, then the k_x, k_y monomials of eqs. delta2b and
//           delta4b are applied and the fields summed into k_z-power groups,
//   z-pass: transform along z, Legendre recombination F_2, F_4 (eqs. F2,
//           delta4), window compensation and shell binning (eq. shell) of
//           |F_0|^2, F_2 F_0*, F_4 F_0*, |F_2|^2.
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

// ----------------------------------------------------------------------------
// x-pass: per grid row (y, z) build the moment fields at the nodes, pack them
// two per complex pencil, FFT along x and unpack the two half-spectra.
// S1 layout: [field][z][y][kx], kx = 0..N/2.
// ----------------------------------------------------------------------------

__global__ void __launch_bounds__(256) k_xpass(const unsigned long long* __restrict__ gridq,
                                               const float* __restrict__ gridf, GeomDev g, MomentTable mt,
                                               FftPlan fp, const float2* __restrict__ tw, float2* __restrict__ S1) {
  extern __shared__ float2 smem[];
  const int N = g.N, NH = g.NH;
  const int npair = (mt.nfields + 1) >> 1;
  float* rowF = reinterpret_cast<float*>(smem);
  float2* A = smem + ((N + 1) >> 1) + 1;
  float2* B = A + npair * N;
  const size_t plane = (size_t)N * NH;
  for (int row = blockIdx.x; row < N * N; row += gridDim.x) {
    const int z = row / N, y = row - z * N;
    const size_t gbase = (size_t)row * N;
    for (int x = threadIdx.x; x < N; x += blockDim.x)
      rowF[x] = gridq ? (float)(long long)gridq[gbase + x] * kFixInvF : gridf[gbase + x];
    __syncthreads();
    const float Y = fmaf((float)y, g.H, g.ry), Z = fmaf((float)z, g.H, g.rz);
    for (int t = threadIdx.x; t < npair * N; t += blockDim.x) {
      const int p = t / N, x = t - p * N;
      float hx[5], hy[5], hz[5];
      if (g.los_inf) {
        hx[1] = g.lx; hy[1] = g.ly; hz[1] = g.lz;
      } else {
        const float X = fmaf((float)x, g.H, g.rx);
        const float r2 = X * X + Y * Y + Z * Z;
        const float inv = r2 > 0.f ? rsqrtf(r2) : 0.f;
        hx[1] = X * inv; hy[1] = Y * inv; hz[1] = Z * inv;
      }
      hx[2] = hx[1] * hx[1]; hx[3] = hx[2] * hx[1]; hx[4] = hx[2] * hx[2];
      hy[2] = hy[1] * hy[1]; hy[3] = hy[2] * hy[1]; hy[4] = hy[2] * hy[2];
      hz[2] = hz[1] * hz[1]; hz[3] = hz[2] * hz[1]; hz[4] = hz[2] * hz[2];
      const float f = rowF[x];
      const int q0 = 2 * p, q1 = 2 * p + 1;
      const float m0 = f * pw(hx, mt.e[q0][0]) * pw(hy, mt.e[q0][1]) * pw(hz, mt.e[q0][2]);
      const float m1 = q1 < mt.nfields ? f * pw(hx, mt.e[q1][0]) * pw(hy, mt.e[q1][1]) * pw(hz, mt.e[q1][2]) : 0.f;
      A[p * N + x] = make_float2(m0, m1);
    }
    __syncthreads();
    const float2* R = fft_smem<-1>(A, B, npair, N, fp, tw);
    for (int t = threadIdx.x; t < npair * NH; t += blockDim.x) {
      const int p = t / NH, k = t - p * NH;
      const float2 zk = R[p * N + k];
      const float2 zm = R[p * N + (k == 0 ? 0 : N - k)];
      const int q0 = 2 * p, q1 = 2 * p + 1;
      const size_t off = ((size_t)z * N + y) * NH + k;
      S1[(size_t)q0 * N * plane + off] = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
      if (q1 < mt.nfields)
        S1[(size_t)q1 * N * plane + off] = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
    }
    __syncthreads();
  }
}

// ----------------------------------------------------------------------------
// y-pass: for a tile of TX consecutive kx at one z, FFT each field along y and
// sum the fields of each k_z-power group with their k_x, k_y monomials.
// S2 layout: [group][z][ky][kx].
// ----------------------------------------------------------------------------

constexpr int kTX = 8;      // kx columns per tile
constexpr int kRuns = 32;   // threads per column
constexpr int kRL = 16;     // max points per thread along the pencil (N <= 512)

__device__ __forceinline__ int signed_mode(int k, int N) { return k <= N / 2 ? k : k - N; }

__global__ void __launch_bounds__(kTX * kRuns) k_ypass(const float2* __restrict__ S1, GeomDev g, MomentTable mt,
                                                       FftPlan fp, const float2* __restrict__ tw,
                                                       float2* __restrict__ S2) {
  extern __shared__ float2 smem[];
  const int N = g.N, NH = g.NH;
  const int pst = N + 1;
  float2* A = smem;
  float2* B = smem + kTX * pst;
  const int z = blockIdx.y;
  const int kx0 = blockIdx.x * kTX;
  const int tw_ = min(kTX, NH - kx0);
  const int c = threadIdx.x % kTX, run = threadIdx.x / kTX;
  const int rl = (N + kRuns - 1) / kRuns;
  const int y0 = run * rl;
  const float nx = (float)(kx0 + c);
  const size_t plane = (size_t)N * NH;
  for (int gi = 0; gi < mt.ngroups; ++gi) {
    float2 acc[kRL];
#pragma unroll
    for (int i = 0; i < kRL; ++i) acc[i] = make_float2(0.f, 0.f);
    for (int m = 0; m < mt.g_nmem[gi]; ++m) {
      const int q = mt.g_field[gi][m];
      const float2* src = S1 + (size_t)q * N * plane + (size_t)z * plane + kx0;
      for (int t = threadIdx.x; t < N * kTX; t += blockDim.x) {
        const int yy = t / kTX, cc = t - yy * kTX;
        A[cc * pst + yy] = cc < tw_ ? src[(size_t)yy * NH + cc] : make_float2(0.f, 0.f);
      }
      __syncthreads();
      const float2* R = fft_smem<-1>(A, B, kTX, pst, fp, tw);
      const float coef = mt.g_coef[gi][m];
      const int ei = mt.g_ei[gi][m], ej = mt.g_ej[gi][m];
      float mx = 1.f;
      for (int e = 0; e < ei; ++e) mx *= nx;
#pragma unroll
      for (int i = 0; i < kRL; ++i) {
        const int ky = y0 + i;
        if (i < rl && ky < N) {
          const float ny = (float)signed_mode(ky, N);
          float my = 1.f;
          for (int e = 0; e < ej; ++e) my *= ny;
          const float s = coef * mx * my;
          const float2 v = R[c * pst + ky];
          acc[i].x = fmaf(s, v.x, acc[i].x);
          acc[i].y = fmaf(s, v.y, acc[i].y);
        }
      }
      __syncthreads();
    }
    if (c < tw_) {
      float2* dst = S2 + (size_t)gi * N * plane + (size_t)z * plane + kx0 + c;
#pragma unroll
      for (int i = 0; i < kRL; ++i) {
        const int ky = y0 + i;
        if (i < rl && ky < N) dst[(size_t)ky * NH] = acc[i];
      }
    }
  }
}

// ----------------------------------------------------------------------------
// z-pass: for a tile of TX consecutive kx at one ky, FFT each group along z,
// recombine F_0, F_2, F_4, compensate and bin.  Each thread owns a run of
// consecutive k_z, along which |n| is monotone, sums a run in FP32 and adds
// it to the block's FP64 bins (shared-memory atomics) only when the bin changes.
// Per-block partials: part[(q * nbins + b) * nblk + blk], counts likewise.
// ----------------------------------------------------------------------------

// MODE 0: P bins.  MODE 1: P bins and export of F_0, F_2, F_4 on the
// bispectrum shells into the compact cube E.  MODE 2 (the w^2-weighted field
// F^w): per-shell sums of Re F_l F^w_0* and Re F_0 F^w_l* (thin-shell shot
// noise of eq. SNbisp2thin) with F_l read back from E.
template <int MODE>
__global__ void __launch_bounds__(kTX * kRuns) k_zpass(const float2* __restrict__ S2, GeomDev g, MomentTable mt,
                                                       FftPlan fp, const float2* __restrict__ tw, ZParams zp,
                                                       double* __restrict__ part, int* __restrict__ partc) {
  extern __shared__ float2 smem[];
  const int N = g.N, NH = g.NH;
  const int pst = N + 1;
  float2* A = smem;
  float2* B = smem + kTX * pst;
  const int nkey = MODE == 2 ? zp.nshells : zp.nbins;
  double* sb = reinterpret_cast<double*>(B + kTX * pst);  // [BQ_N][nkey]
  int* sc = reinterpret_cast<int*>(sb + BQ_N * nkey);
  for (int t = threadIdx.x; t < BQ_N * nkey; t += blockDim.x) sb[t] = 0.0;
  for (int t = threadIdx.x; t < nkey; t += blockDim.x) sc[t] = 0;
  const int ky = blockIdx.y;
  const int kx0 = blockIdx.x * kTX;
  const int tw_ = min(kTX, NH - kx0);
  const int c = threadIdx.x % kTX, run = threadIdx.x / kTX;
  const int rl = (N + kRuns - 1) / kRuns;
  const int z0 = run * rl;
  const size_t plane = (size_t)N * NH;
  float2 f0[kRL], s2[kRL], s4[kRL];
#pragma unroll
  for (int i = 0; i < kRL; ++i) {
    f0[i] = make_float2(0.f, 0.f);
    s2[i] = f0[i];
    s4[i] = f0[i];
  }
  for (int gi = 0; gi < mt.ngroups; ++gi) {
    const float2* src = S2 + (size_t)gi * N * plane + (size_t)ky * NH + kx0;
    for (int t = threadIdx.x; t < N * kTX; t += blockDim.x) {
      const int zz = t / kTX, cc = t - zz * kTX;
      A[cc * pst + zz] = cc < tw_ ? src[(size_t)zz * plane + cc] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const float2* R = fft_smem<-1>(A, B, kTX, pst, fp, tw);
    const int ell = mt.g_ell[gi], p = mt.g_p[gi];
#pragma unroll
    for (int i = 0; i < kRL; ++i) {
      const int kz = z0 + i;
      if (i < rl && kz < N) {
        const float2 v = R[c * pst + kz];
        if (ell == 0) {
          f0[i] = v;
        } else {
          const float nz = (float)signed_mode(kz, N);
          float mz = 1.f;
          for (int e = 0; e < p; ++e) mz *= nz;
          if (ell == 2) {
            s2[i].x = fmaf(mz, v.x, s2[i].x);
            s2[i].y = fmaf(mz, v.y, s2[i].y);
          } else {
            s4[i].x = fmaf(mz, v.x, s4[i].x);
            s4[i].y = fmaf(mz, v.y, s4[i].y);
          }
        }
      }
    }
    __syncthreads();
  }
  // recombination and binning
  const int kx = kx0 + c;
  const bool colok = c < tw_ && kx < N / 2;
  const int nyv = signed_mode(ky, N);
  const bool rowok = !(ky == N / 2);
  const float wcol = kx == 0 ? 1.f : 2.f;
  const float wxy = colok ? zp.winv[kx] * zp.winv[N + ky] : 0.f;
  int curb = -1, cnt = 0;
  float acc[BQ_N];
#pragma unroll
  for (int q = 0; q < BQ_N; ++q) acc[q] = 0.f;
#pragma unroll
  for (int i = 0; i < kRL; ++i) {
    const int kz = z0 + i;
    int b = -1;
    float vals[BQ_N];
    if (colok && rowok && i < rl && kz < N && kz != N / 2) {
      const int nzv = signed_mode(kz, N);
      const int n2 = kx * kx + nyv * nyv + nzv * nzv;
      const int sh = (MODE != 0 && n2 < zp.nsh2) ? (int)zp.slut[n2] : -1;
      b = MODE == 2 ? sh : (n2 > 0 ? zp.lut[n2] : -1);
      if (b >= 0 || sh >= 0) {
        const float wc = wxy * zp.winv[2 * N + kz];
        const float fn2 = (float)n2;
        const float2 F0 = make_float2(f0[i].x * wc, f0[i].y * wc);
        float2 F2 = make_float2(0.f, 0.f), F4 = make_float2(0.f, 0.f);
        if (zp.lmax >= 2) {
          const float i2 = 1.0f / fn2;
          F2 = make_float2(wc * (1.5f * s2[i].x * i2 - 0.5f * f0[i].x), wc * (1.5f * s2[i].y * i2 - 0.5f * f0[i].y));
          if (zp.lmax >= 4) {
            const float i4 = i2 * i2;
            F4 = make_float2(4.375f * wc * s4[i].x * i4 - 2.5f * F2.x - 0.875f * F0.x,
                             4.375f * wc * s4[i].y * i4 - 2.5f * F2.y - 0.875f * F0.y);
          }
        }
        if (MODE != 2) {
          vals[BQ_K] = zp.kf * sqrtf(fn2);
          vals[BQ_F00] = F0.x * F0.x + F0.y * F0.y;
          vals[BQ_F20] = F2.x * F0.x + F2.y * F0.y;
          vals[BQ_F40] = F4.x * F0.x + F4.y * F0.y;
          vals[BQ_F22] = F2.x * F2.x + F2.y * F2.y;
        }
        if (MODE != 0 && sh >= 0) {
          const int w2 = 2 * zp.mm + 1;
          const size_t e = ((size_t)(nzv + zp.mm) * w2 + (nyv + zp.mm)) * (zp.mm + 1) + kx;
          const size_t es = (size_t)w2 * w2 * (zp.mm + 1);
          if (MODE == 1) {
            zp.E[e] = F0;
            zp.E[es + e] = F2;
            zp.E[2 * es + e] = F4;
          } else {
            // here F0, F2, F4 are the Legendre fields of F^w; E holds those of F
            const float2 E0 = zp.E[e], E2 = zp.E[es + e], E4 = zp.E[2 * es + e];
            vals[SQ_00] = E0.x * F0.x + E0.y * F0.y;
            vals[SQ_20] = E2.x * F0.x + E2.y * F0.y;
            vals[SQ_40] = E4.x * F0.x + E4.y * F0.y;
            vals[SQ_02] = E0.x * F2.x + E0.y * F2.y;
            vals[SQ_04] = E0.x * F4.x + E0.y * F4.y;
          }
        }
      }
    }
    if (b != curb) {
      if (curb >= 0) {
        atomicAdd(sc + curb, cnt);
#pragma unroll
        for (int q = 0; q < BQ_N; ++q) atomicAdd(sb + q * nkey + curb, (double)acc[q]);
      }
      curb = b;
      cnt = 0;
#pragma unroll
      for (int q = 0; q < BQ_N; ++q) acc[q] = 0.f;
    }
    if (b >= 0) {
      cnt += (int)wcol;
#pragma unroll
      for (int q = 0; q < BQ_N; ++q) acc[q] = fmaf(wcol, vals[q], acc[q]);
    }
  }
  if (curb >= 0) {
    atomicAdd(sc + curb, cnt);
#pragma unroll
    for (int q = 0; q < BQ_N; ++q) atomicAdd(sb + q * nkey + curb, (double)acc[q]);
  }
  __syncthreads();
  const int blk = blockIdx.y * gridDim.x + blockIdx.x;
  const int nblk = gridDim.x * gridDim.y;
  for (int t = threadIdx.x; t < BQ_N * nkey; t += blockDim.x) part[(size_t)t * nblk + blk] = sb[t];
  for (int t = threadIdx.x; t < nkey; t += blockDim.x) partc[(size_t)t * nblk + blk] = sc[t];
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

size_t xpass_smem(int N, int nfields) { return sizeof(float2) * (((N + 1) / 2) + 1 + 2 * ((nfields + 1) / 2) * N); }
size_t yz_smem(int N) { return sizeof(float2) * 2 * kTX * (N + 1); }
size_t zpass_smem(int N, int nbins) { return yz_smem(N) + sizeof(double) * BQ_N * nbins + sizeof(int) * nbins; }
int yz_tiles(int N) { return (N / 2 + 1 + kTX - 1) / kTX; }

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

cudaError_t launch_xpass(const unsigned long long* gq, const float* gf, const GeomDev& g, const MomentTable& mt,
                         const FftPlan& fp, const float2* tw, float2* S1, int nsm, cudaStream_t s) {
  const size_t sm = xpass_smem(g.N, mt.nfields);
  cudaFuncSetAttribute(k_xpass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  int occ = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_xpass, 256, sm);
  int grid = nsm * (occ > 0 ? occ : 1);
  if (grid > g.N * g.N) grid = g.N * g.N;
  k_xpass<<<grid, 256, sm, s>>>(gq, gf, g, mt, fp, tw, S1);
  return cudaGetLastError();
}

cudaError_t launch_ypass(const float2* S1, const GeomDev& g, const MomentTable& mt, const FftPlan& fp,
                         const float2* tw, float2* S2, cudaStream_t s) {
  const size_t sm = yz_smem(g.N);
  cudaFuncSetAttribute(k_ypass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  dim3 grid(yz_tiles(g.N), g.N);
  k_ypass<<<grid, kTX * kRuns, sm, s>>>(S1, g, mt, fp, tw, S2);
  return cudaGetLastError();
}

cudaError_t launch_zpass(const float2* S2, const GeomDev& g, const MomentTable& mt, const FftPlan& fp,
                         const float2* tw, const ZParams& zp, double* part, int* partc, cudaStream_t s) {
  const size_t sm = zpass_smem(g.N, zp.mode == 2 ? zp.nshells : zp.nbins);
  dim3 grid(yz_tiles(g.N), g.N);
  if (zp.mode == 0) {
    cudaFuncSetAttribute(k_zpass<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_zpass<0><<<grid, kTX * kRuns, sm, s>>>(S2, g, mt, fp, tw, zp, part, partc);
  } else if (zp.mode == 1) {
    cudaFuncSetAttribute(k_zpass<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_zpass<1><<<grid, kTX * kRuns, sm, s>>>(S2, g, mt, fp, tw, zp, part, partc);
  } else {
    cudaFuncSetAttribute(k_zpass<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_zpass<2><<<grid, kTX * kRuns, sm, s>>>(S2, g, mt, fp, tw, zp, part, partc);
  }
  return cudaGetLastError();
}

cudaError_t launch_reduce_bins(const double* part, const int* partc, int nblk, int nbins, double* out, long long* outc,
                               cudaStream_t s) {
  k_reduce_bins<<<(BQ_N + 1) * nbins, 256, 0, s>>>(part, partc, nblk, nbins, out, outc);
  return cudaGetLastError();
}

}  // namespace fkp
