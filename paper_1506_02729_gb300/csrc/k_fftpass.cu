// k_fftpass.cu - the three FFT passes of the power-spectrum path.
//
//   x-pass  per grid row (blocks walk rows, the next row's values loaded
//           while this one is transformed): moment fields F x^_a x^_b (...)
//           built at the nodes about the observer (eqs. Qij, Qijkl, Qab), two
//           real fields packed per complex pencil (XOR-swizzled interleave),
//           FFT along x, unpacked into half spectra.
//   y-pass  per (z, k_x tile): FFT of each field along y, then the k_x, k_y
//           polynomials of eqs. delta2b and delta4b (with the multinomial
//           multiplicities and the trace identities of the unit vector x^),
//           summed into k_z-power groups.
//   z-pass  per (k_y, k_x tile), persistent blocks walking their tiles with
//           the next tile's first copy in flight: FFT of each group along z, Legendre
//           recombination F_2 = 3/2 S_2/|n|^2 - F_0/2 and
//           F_4 = 35/8 S_4/|n|^4 - 5/2 F_2 - 7/8 F_0 (eqs. F2, delta4),
//           window compensation and shell binning (eq. shell).
//
// Block shapes and the x-pass grid are chosen per grid by timing when a plan
// is made (PassSchedule).  Layouts are tile-major so that every tile a pass
// reads is one contiguous block, fetched with a bulk (TMA) copy while the
// previous one is being transformed:
//   S1[field][z][xt][y][c]   (k_x = 8 xt + c), written by the x-pass
//   S2[group][xt][ky][z][c]  written by the y-pass, read by the z-pass
#include <cuda_runtime.h>
#include <stdint.h>

#include "fkp_internal.h"

namespace fkp {

constexpr int kT = 8;        // k_x columns per tile (64 bytes of complex64)
// y-pass blocks (8, 32), two per SM; z-pass blocks (8, 64), one per SM (its
// three accumulators per point need the registers)
// The y- and z-pass blocks are (8, NT / 8): NT / 8 threads per column, each
// holding RL = 512 / (NT / 8) points (N <= 512).  NT is 256 or 512, chosen per
// grid by timing when a plan is made (PassSchedule).
template <int NT>
struct PassShape {
  static constexpr int kRun = NT / kT;
  static constexpr int kRL = (512 + kRun - 1) / kRun;
  static constexpr int kMinBlocks = NT <= 256 ? 2 : 1;
};

__device__ __forceinline__ int smode(int k, int N) { return k <= N / 2 ? k : k - N; }

__device__ __forceinline__ float powi(float v, int e) {
  float r = 1.f;
  for (int i = 0; i < e; ++i) r *= v;
  return r;
}

__device__ __forceinline__ float pw5(const float* h, int e) {
  return e == 0 ? 1.f : (e == 1 ? h[1] : (e == 2 ? h[2] : (e == 3 ? h[3] : h[4])));
}

// ----------------------------------------------------------------------------
// x-pass
// ----------------------------------------------------------------------------

// Moment-field exponents (i, j, k) of x^_x^i x^_y^j x^_z^k in the order the
// host's moment table uses: F_0; for ell = 2, 4 the components with z power
// p = 0, 1 (j ascending); then zzzz (the trace-reduced set: 1 + 5 + 10).
__host__ __device__ constexpr int nfields_of(int lmax) { return lmax >= 4 ? 16 : (lmax >= 2 ? 6 : 1); }
__host__ __device__ constexpr int field_exp(int q, int a) {
  int idx = 0;
  for (int ell = 0; ell <= 4; ell += 2) {
    for (int p = 0; p <= (ell ? 1 : 0); ++p)
      for (int j = 0; j <= ell - p; ++j) {
        if (idx == q) return a == 0 ? ell - p - j : (a == 1 ? j : p);
        ++idx;
      }
    if (ell == 4 && idx == q) return a == 2 ? 4 : 0;
  }
  return 0;
}

// Moment values of pencil pairs P.., packed two real fields per complex value;
// template recursion keeps every exponent a compile-time constant.
template <int NP, int NF, int P, bool SWZ>
__device__ __forceinline__ void build_pairs(float f, const float (&hx)[5], const float (&hy)[5], const float (&hz)[5],
                                            float2* A, int x) {
  if constexpr (P < NP) {
    constexpr int a0 = field_exp(2 * P, 0), b0 = field_exp(2 * P, 1), c0 = field_exp(2 * P, 2);
    constexpr int a1 = field_exp(2 * P + 1, 0), b1 = field_exp(2 * P + 1, 1), c1 = field_exp(2 * P + 1, 2);
    const float m0 = f * hx[a0] * hy[b0] * hz[c0];
    const float m1 = (2 * P + 1 < NF) ? f * hx[a1] * hy[b1] * hz[c1] : 0.f;
    A[ilv<NP, SWZ>(x, P)] = make_float2(m0, m1);
    build_pairs<NP, NF, P + 1, SWZ>(f, hx, hy, hz, A, x);
  }
}

// Block (NP, 32): threadIdx.x is the packed pencil (pair of fields) in the
// FFT; a radix-R stage's N/R butterflies per pencil are strided over
// threadIdx.y, so no index is divided by NP.  The register cap keeps as many
// blocks per SM as shared memory allows for the full moment set (4 up to
// N = 256, 3 above).
template <int N_, int LMAX>
__global__ void __launch_bounds__(32 * ((nfields_of(LMAX) + 1) / 2), LMAX < 4 ? 1 : (N_ > 0 && N_ <= 256 ? 4 : 3))
    k_xpass2(
    const unsigned long long* __restrict__ gq, const float* __restrict__ gf, GeomDev g, FftPlan fp,
    const float2* __restrict__ twg, float2* __restrict__ S1, MockBatch mb) {
  if (gq) gq += (long long)blockIdx.z * mb.in;
  if (gf) gf += (long long)blockIdx.z * mb.in;
  S1 += (long long)blockIdx.z * mb.out;
  constexpr int NF = nfields_of(LMAX);
  constexpr int NP = (NF + 1) / 2;
  constexpr int NTX = 32 * NP;
  // swizzled interleave when NP is a power of two: the moment stores (one
  // pencil slot, consecutive x) and the unpack loads (consecutive k) are then
  // free of bank conflicts
  constexpr bool SWZ = NP > 1 && (NP & (NP - 1)) == 0;
  extern __shared__ float2 sm[];
  const int N = N_ ? N_ : g.N;
  const int NH = N / 2 + 1, NXT = (NH + kT - 1) / kT;
  const int tid = threadIdx.y * NP + threadIdx.x;
  float2* tw = sm;
  float* rowF = reinterpret_cast<float*>(sm + N);
  float2* A = sm + N + N / 2;
  float2* B = A + NP * N;
  for (int i = tid; i < N; i += NTX) tw[i] = twg[i];
  const size_t fsz = (size_t)N * NXT * N * kT;
  // the next row's grid values are loaded into registers while this row is
  // transformed (N <= 512)
  constexpr int NPRE = (512 + NTX - 1) / NTX;
  float pre[NPRE];
  auto load_row = [&](int row) {
#pragma unroll
    for (int j = 0; j < NPRE; ++j) {
      const int x = tid + j * NTX;
      float v = 0.f;
      if (row < N * N && x < N) {
        const size_t gi = (size_t)row * N + x;
        v = gq ? (float)(long long)__ldg(gq + gi) * kFixInvF : __ldg(gf + gi);
      }
      pre[j] = v;
    }
  };
  load_row(blockIdx.x);
  for (int row = blockIdx.x; row < N * N; row += gridDim.x) {
    const int z = row / N, y = row - z * N;
#pragma unroll
    for (int j = 0; j < NPRE; ++j) {
      const int x = tid + j * NTX;
      if (x < N) rowF[x] = pre[j];
    }
    load_row(row + gridDim.x);
    __syncthreads();
    const float Y = fmaf((float)y, g.H, g.ry), Z = fmaf((float)z, g.H, g.rz);
    for (int x = tid; x < N; x += NTX) {
      float hx[5], hy[5], hz[5];
      if (g.los_inf) {
        hx[1] = g.lx; hy[1] = g.ly; hz[1] = g.lz;
      } else {
        const float X = fmaf((float)x, g.H, g.rx);
        const float r2 = X * X + Y * Y + Z * Z;
        const float inv = r2 > 0.f ? rsqrtf(r2) : 0.f;
        hx[1] = X * inv; hy[1] = Y * inv; hz[1] = Z * inv;
      }
      hx[0] = hy[0] = hz[0] = 1.f;
      hx[2] = hx[1] * hx[1]; hx[3] = hx[2] * hx[1]; hx[4] = hx[2] * hx[2];
      hy[2] = hy[1] * hy[1]; hy[3] = hy[2] * hy[1]; hy[4] = hy[2] * hy[2];
      hz[2] = hz[1] * hz[1]; hz[3] = hz[2] * hz[1]; hz[4] = hz[2] * hz[2];
      build_pairs<NP, NF, 0, SWZ>(rowF[x], hx, hy, hz, A, x);
    }
    __syncthreads();
    const float2* R = fft_any<N_, NP, NTX, -1, SWZ>(A, B, fp, tw);
    // unpack: consecutive threads take consecutive k_x of one field, so the
    // stores into the tile-major layout are 64-byte contiguous runs
    const int ncol = NXT * kT;
    for (int t = tid; t < NP * ncol; t += NTX) {
      const int p = t / ncol, k = t - p * ncol;
      float2 o0 = make_float2(0.f, 0.f), o1 = o0;
      if (k < NH) {
        const float2 zk = R[ilv<NP, SWZ>(k, p)];
        const float2 zm = R[ilv<NP, SWZ>(k == 0 ? 0 : N - k, p)];
        o0 = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
        o1 = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
      }
      const size_t off = (((size_t)z * NXT + (k >> 3)) * N + y) * kT + (k & 7);
      S1[(size_t)(2 * p) * fsz + off] = o0;
      if (2 * p + 1 < NF) S1[(size_t)(2 * p + 1) * fsz + off] = o1;
    }
    __syncthreads();
  }
}

// ----------------------------------------------------------------------------
// y-pass
// ----------------------------------------------------------------------------

// Block (8, 32): threadIdx.x is the k_x column of the tile (the FFT pencil);
// thread (c, r) accumulates k_y = r, r + 32, r + 64, ... (a warp's four r
// read 32 consecutive values: no bank conflicts).  The fields are read
// sweep by sweep; a sweep accumulates up to two output groups, each member
// with a polynomial coefficient in n_y evaluated by Horner's rule.
template <int N_, int NT>
__global__ void __launch_bounds__(NT, PassShape<NT>::kMinBlocks) k_ypass2(const float2* __restrict__ S1,
                                                   const unsigned long long* __restrict__ gq,
                                                   const float* __restrict__ gf, GeomDev g, MomentTable mt,
                                                   FftPlan fp, const float2* __restrict__ twg,
                                                   float2* __restrict__ S2, int* __restrict__ err, MockBatch mb) {
  S1 += (long long)blockIdx.z * mb.in;
  if (gq) gq += (long long)blockIdx.z * mb.in2;
  if (gf) gf += (long long)blockIdx.z * mb.in2;
  S2 += (long long)blockIdx.z * mb.out;
  extern __shared__ __align__(128) unsigned char smraw[];
  const int N = N_ ? N_ : g.N;
  const int NH = N / 2 + 1, NXT = (NH + kT - 1) / kT;
  const int tile = N * kT;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smraw);
  float2* buf0 = reinterpret_cast<float2*>(smraw + 128);
  float2* buf1 = buf0 + tile;
  float2* work = buf1 + tile;
  float2* tw = work + tile;
  const int xt = blockIdx.x, z = blockIdx.y;
  const size_t fsz = (size_t)N * NXT * N * kT;
  const size_t gsz = fsz;
  const uint32_t bytes = (uint32_t)(tile * sizeof(float2));
  const int tid = threadIdx.y * kT + threadIdx.x;
  for (int i = tid; i < N; i += NT) tw[i] = twg[i];
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
  int total = 0;
  for (int s = 0; s < mt.nsweeps; ++s) total += mt.s_nmem[s];
  auto src_of = [&](int q) { return S1 + (size_t)q * fsz + ((size_t)z * NXT + xt) * tile; };
  if (tid == 0) {
    mbar_expect_tx(&bar[0], bytes);
    tma_load_1d(buf0, src_of(mt.s_field[0][0]), bytes, &bar[0]);
  }
  const int c = threadIdx.x, run = threadIdx.y;
  const int rl = (N + PassShape<NT>::kRun - 1) / PassShape<NT>::kRun;
  const int kx = xt * kT + c;
  const float nx = (float)kx;
  int it = 0;
  for (int sw = 0; sw < mt.nsweeps; ++sw) {
    const int nout = mt.s_nout[sw];
    float2 acc0[PassShape<NT>::kRL], acc1[PassShape<NT>::kRL];
#pragma unroll
    for (int i = 0; i < PassShape<NT>::kRL; ++i) {
      acc0[i] = make_float2(0.f, 0.f);
      acc1[i] = acc0[i];
    }
    for (int m = 0; m < mt.s_nmem[sw]; ++m, ++it) {
      const int cur = it & 1;
      float2* bc = cur ? buf1 : buf0;
      if (tid == 0 && it + 1 < total) {
        int s2 = sw, m2 = m + 1;
        if (m2 == mt.s_nmem[sw]) { s2 = sw + 1; m2 = 0; }
        fence_proxy_async();
        mbar_expect_tx(&bar[cur ^ 1], bytes);
        tma_load_1d(cur ? buf0 : buf1, src_of(mt.s_field[s2][m2]), bytes, &bar[cur ^ 1]);
      }
      mbar_wait(&bar[cur], (uint32_t)((it >> 1) & 1), err, 4);
      const float2* R = fft_any<N_, kT, NT, -1>(bc, work, fp, tw);
      // coefficients a[o][j] of n_y^j for this member and column
      float a[2][5];
#pragma unroll
      for (int o = 0; o < 2; ++o)
#pragma unroll
        for (int j = 0; j < 5; ++j) {
          float v = 0.f;
#pragma unroll
          for (int t = 0; t < 2; ++t)
            if (mt.s_j[sw][m][o][t] == j) v += mt.s_c[sw][m][o][t] * powi(nx, mt.s_i[sw][m][o][t]);
          a[o][j] = v;
        }
#pragma unroll
      for (int i = 0; i < PassShape<NT>::kRL; ++i) {
        const int ky = i * PassShape<NT>::kRun + run;
        if (i < rl && ky < N) {
          const float ny = (float)smode(ky, N);
          const float2 v = R[ky * kT + c];
          const float s0 = fmaf(fmaf(fmaf(fmaf(a[0][4], ny, a[0][3]), ny, a[0][2]), ny, a[0][1]), ny, a[0][0]);
          acc0[i].x = fmaf(s0, v.x, acc0[i].x);
          acc0[i].y = fmaf(s0, v.y, acc0[i].y);
          if (nout > 1) {
            const float s1 = fmaf(fmaf(fmaf(fmaf(a[1][4], ny, a[1][3]), ny, a[1][2]), ny, a[1][1]), ny, a[1][0]);
            acc1[i].x = fmaf(s1, v.x, acc1[i].x);
            acc1[i].y = fmaf(s1, v.y, acc1[i].y);
          }
        }
      }
      __syncthreads();
    }
    // the observer's node (x^ = 0): its F, x- and y-transformed, joins T
    if (mt.s_obs[sw] >= 0 && z == g.obs_z) {
      const size_t node = ((size_t)g.obs_z * N + g.obs_y) * N + g.obs_x;
      const float fo = gq ? (float)(long long)gq[node] * kFixInvF : gf[node];
#pragma unroll
      for (int i = 0; i < PassShape<NT>::kRL; ++i) {
        const int ky = i * PassShape<NT>::kRun + run;
        if (i < rl && ky < N) {
          const int ph = (int)(((long long)kx * g.obs_x + (long long)ky * g.obs_y) % N);
          float sn, cs;
          sincospif(-2.0f * (float)ph / (float)N, &sn, &cs);
          float2& t = mt.s_obs[sw] ? acc1[i] : acc0[i];
          t.x = fmaf(fo, cs, t.x);
          t.y = fmaf(fo, sn, t.y);
        }
      }
    }
#pragma unroll
    for (int o = 0; o < 2; ++o) {
      if (o >= nout) break;
      float2* dst = S2 + (size_t)mt.s_out[sw][o] * gsz + (size_t)xt * N * tile + (size_t)z * kT + c;
#pragma unroll
      for (int i = 0; i < PassShape<NT>::kRL; ++i) {
        const int ky = i * PassShape<NT>::kRun + run;
        if (i < rl && ky < N) dst[(size_t)ky * tile] = o ? acc1[i] : acc0[i];
      }
    }
  }
}

// ----------------------------------------------------------------------------
// k_z-power groups as the z-pass applies them (the host's moment table lists
// the same values; moments_match checks them): group g adds to F_0 (zg_f0),
// zg_c2 nz^zg_p2 times itself to S_2 and zg_c4 nz^zg_p4 times itself to S_4.
// ----------------------------------------------------------------------------

__host__ __device__ constexpr int zg_f0(int g) { return g == 0 ? 1 : 0; }
__host__ __device__ constexpr float zg_c2(int g) {
  return g == 0 ? 1.f : (g == 1 ? 1.f : (g == 2 ? -1.f : (g == 3 ? 1.f : 0.f)));
}
__host__ __device__ constexpr int zg_p2(int g) { return g == 0 ? 2 : (g == 2 ? 2 : (g == 3 ? 1 : 0)); }
__host__ __device__ constexpr float zg_c4(int g) {
  return g == 1 ? 6.f : (g == 3 ? 2.f : (g == 4 || g == 6 || g == 8 ? 1.f : (g == 5 || g == 7 ? -1.f : 0.f)));
}
__host__ __device__ constexpr int zg_p4(int g) {
  return g == 1 || g == 5 ? 2 : (g == 3 || g == 7 ? 3 : (g == 6 ? 1 : (g == 8 ? 4 : 0)));
}

// v^e for e in 0..4 from v and v^2, by selection (no loop).
__device__ __forceinline__ float pwsel(float v, float v2, int e) {
  return e == 0 ? 1.f : (e == 1 ? v : (e == 2 ? v2 : (e == 3 ? v2 * v : v2 * v2)));
}

// One group's contribution to the thread's run of k_z: F_0 (F0), c2 nz^p2 to
// S_2 (A2), c4 nz^p4 to S_4 (A4).
template <int RL, bool F0, bool A2, bool A4, bool PH>
__device__ __forceinline__ void zgroup(const float2* R, int z0, int rl, int N, int c, float c2, int p2, float c4,
                                       int p4, float2 (&f0)[RL], float2 (&s2)[RL], float2 (&s4)[RL],
                                       const float2* ph, float2 phxy) {
#pragma unroll
  for (int i = 0; i < RL; ++i) {
    const int kz = z0 + i;
    if (i < rl && kz < N) {
      float2 v = R[kz * kT + c];
      if (PH) v = cmul(v, cmul(phxy, ph[kz]));
      const float nz = (float)smode(kz, N), nz2 = nz * nz;
      if (F0) f0[i] = cadd(f0[i], v);
      if (A2) {
        const float m = c2 * pwsel(nz, nz2, p2);
        s2[i].x = fmaf(m, v.x, s2[i].x);
        s2[i].y = fmaf(m, v.y, s2[i].y);
      }
      if (A4) {
        const float m = c4 * pwsel(nz, nz2, p4);
        s4[i].x = fmaf(m, v.x, s4[i].x);
        s4[i].y = fmaf(m, v.y, s4[i].y);
      }
    }
  }
}

// ----------------------------------------------------------------------------
// z-pass (MODE 0: P bins; 1: P bins + export on the shells; 2: F^w shell sums)
// ----------------------------------------------------------------------------

// Block (8, 64): threadIdx.x is the k_x column, threadIdx.y the run of k_z.
// The epilogue walks each thread's run of consecutive k_z (|n| is monotone
// along it), sums a run in FP32 and adds it to the tile's fixed-point bins
// in shared memory when the bin changes (integer adds: the result does not
// depend on the order of the threads); each tile's bins join the block's
// FP64 sums in tile order, and blocks' bins are reduced in FP64 in a fixed
// order, so the bins are bit-reproducible for a given launch shape.
template <int N_, int MODE, int NT>
__global__ void __launch_bounds__(NT, PassShape<NT>::kMinBlocks) k_zpass2(const float2* __restrict__ S2, GeomDev g, MomentTable mt,
                                                   FftPlan fp, const float2* __restrict__ twg, ZParams zp,
                                                   double* __restrict__ part, int* __restrict__ partc,
                                                   int* __restrict__ err, MockBatch mb) {
  S2 += (long long)blockIdx.z * mb.in;
  part += (long long)blockIdx.z * mb.out;
  partc += (long long)blockIdx.z * mb.out2;
  extern __shared__ __align__(128) unsigned char smraw[];
  const int N = N_ ? N_ : g.N;
  const int NH = N / 2 + 1, NXT = (NH + kT - 1) / kT;
  const int tile = N * kT;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smraw);
  float2* buf0 = reinterpret_cast<float2*>(smraw + 128);
  float2* buf1 = buf0 + tile;
  float2* work = buf1 + tile;
  float2* tw = work + tile;
  const int nkey = MODE == 2 ? zp.nshells : zp.nbins;
  float2* zph = tw + N;                                   // [N] z half-cell phases (interlaced pairs)
  double* sbd = reinterpret_cast<double*>(zph + N);       // [BQ_N][nkey] the block's FP64 sums over its tiles
  long long* sbi = reinterpret_cast<long long*>(sbd + BQ_N * nkey);  // [BQ_N][nkey] one tile's fixed-point sums
  int* sc = reinterpret_cast<int*>(sbi + BQ_N * nkey);
  unsigned* tmax = reinterpret_cast<unsigned*>(sc + nkey);  // the tile's bound on |value| (FP32 bits)
  const int tid = threadIdx.y * kT + threadIdx.x;
  const int ntiles = NXT * N;
  const size_t gsz = (size_t)N * NXT * N * kT;
  const uint32_t bytes = (uint32_t)(tile * sizeof(float2));
  for (int i = tid; i < N; i += NT) {
    tw[i] = twg[i];
    zph[i] = zp.interlace ? zp.hph[i] : make_float2(1.f, 0.f);
  }
  const int ngt = zp.interlace ? 2 * mt.ngroups : mt.ngroups;  // groups read per tile
  // bin quantities accumulated: the five of P_0..P_4b (or the F^w shell
  // products), and Re F_4 F_2*, |F_4|^2 when the split l = 6, 8 are wanted
  const int nq = MODE == 2 ? SQ_04 + 1 : (zp.split68 ? BQ_N : BQ_F22 + 1);
  for (int t = tid; t < BQ_N * nkey; t += NT) {
    sbi[t] = 0;
    sbd[t] = 0.0;
  }
  for (int t = tid; t < nkey; t += NT) sc[t] = 0;
  if (tid == 0) *tmax = 0u;
  // fixed-point exponent of the k sums: k <= kf sqrt(3) N/2 < kf N
  int ek;
  frexpf(zp.kf * (float)N, &ek);
  const int sk = 49 - ek;
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
  // tile t = (xt, ky) = (t % NXT, t / NXT); group gi of tile t
  auto src_of = [&](int t, int gi) {
    return S2 + (size_t)gi * gsz + ((size_t)(t % NXT) * N + t / NXT) * tile;
  };
  if (tid == 0 && (int)blockIdx.x < ntiles) {
    mbar_expect_tx(&bar[0], bytes);
    tma_load_1d(buf0, src_of(blockIdx.x, 0), bytes, &bar[0]);
  }
  const int c = threadIdx.x, run = threadIdx.y;
  const int rl = (N + PassShape<NT>::kRun - 1) / PassShape<NT>::kRun;
  const int z0 = run * rl;
  // persistent: the block walks its tiles; the copy of the next (tile, group)
  // is always in flight, across tile boundaries too (it counts them: buffer
  // it & 1, phase (it >> 1) & 1)
  int it = 0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
  const int xt = t % NXT, ky = t / NXT;
  float2 f0[PassShape<NT>::kRL], s2[PassShape<NT>::kRL], s4[PassShape<NT>::kRL];
#pragma unroll
  for (int i = 0; i < PassShape<NT>::kRL; ++i) {
    f0[i] = make_float2(0.f, 0.f);
    s2[i] = f0[i];
    s4[i] = f0[i];
  }
  for (int gi = 0; gi < ngt; ++gi, ++it) {
    const int cur = it & 1;
    float2* bc = cur ? buf1 : buf0;
    if (tid == 0) {
      const int tn = gi + 1 < ngt ? t : t + (int)gridDim.x;
      const int gn = gi + 1 < ngt ? gi + 1 : 0;
      if (tn < ntiles) {
        fence_proxy_async();
        mbar_expect_tx(&bar[cur ^ 1], bytes);
        tma_load_1d(cur ? buf0 : buf1, src_of(tn, gn), bytes, &bar[cur ^ 1]);
      }
    }
    mbar_wait(&bar[cur], (uint32_t)((it >> 1) & 1), err, 8);
    const float2* R = fft_any<N_, kT, NT, -1>(bc, work, fp, tw);
    const int gg = gi < mt.ngroups ? gi : gi - mt.ngroups;  // the group's coefficients
    // second grid of an interlaced pair: its half-cell phase
    // e^{-i pi (n_x + n_y + n_z)/N}, the n_x, n_y part fixed per thread
    const float2 phxy = gi < mt.ngroups ? make_float2(1.f, 0.f)
                                        : cmul(zph[(t % NXT) * kT + c < N ? (t % NXT) * kT + c : 0], zph[t / NXT]);
    const int p2 = mt.g_p2[gg], p4 = mt.g_p4[gg];
    const float c2 = mt.g_c2[gg], c4 = mt.g_c4[gg];
    constexpr int RLc = PassShape<NT>::kRL;
    if (gi < mt.ngroups) {
      if (mt.g_f0[gg]) zgroup<RLc, true, true, false, false>(R, z0, rl, N, c, c2, p2, c4, p4, f0, s2, s4, zph, phxy);
      else if (c2 != 0.f && c4 != 0.f) zgroup<RLc, false, true, true, false>(R, z0, rl, N, c, c2, p2, c4, p4, f0, s2, s4, zph, phxy);
      else if (c2 != 0.f) zgroup<RLc, false, true, false, false>(R, z0, rl, N, c, c2, p2, c4, p4, f0, s2, s4, zph, phxy);
      else zgroup<RLc, false, false, true, false>(R, z0, rl, N, c, c2, p2, c4, p4, f0, s2, s4, zph, phxy);
    } else {  // second grid of an interlaced pair: its z half-cell phase
      if (mt.g_f0[gg]) zgroup<RLc, true, true, false, true>(R, z0, rl, N, c, c2, p2, c4, p4, f0, s2, s4, zph, phxy);
      else if (c2 != 0.f && c4 != 0.f) zgroup<RLc, false, true, true, true>(R, z0, rl, N, c, c2, p2, c4, p4, f0, s2, s4, zph, phxy);
      else if (c2 != 0.f) zgroup<RLc, false, true, false, true>(R, z0, rl, N, c, c2, p2, c4, p4, f0, s2, s4, zph, phxy);
      else zgroup<RLc, false, false, true, true>(R, z0, rl, N, c, c2, p2, c4, p4, f0, s2, s4, zph, phxy);
    }
    __syncthreads();
  }
  const int kx = xt * kT + c;
  const bool colok = kx < N / 2;
  const int nyv = smode(ky, N);
  const bool rowok = ky != N / 2;
  const float wcol = kx == 0 ? 1.f : 2.f;
  const float wxy = colok ? zp.scale * zp.winv[kx] * zp.winv[N + ky] : 0.f;
  // Bin sums are made order independent (bit-reproducible): each thread's
  // runs are summed in FP32 in k_z order, then added to the tile's sums as
  // 64-bit fixed-point integers at a scale 2^st set by a bound M on every
  // |value| of the tile (|Re a b*| <= max(|a|^2, |b|^2)), so that a tile's bin
  // sum stays below 2^62; integer adds commute.  First pass: the bound.
  float mloc = 0.f;
#pragma unroll
  for (int i = 0; i < PassShape<NT>::kRL; ++i) {
    const int kz = z0 + i;
    if (colok && rowok && i < rl && kz < N && kz != N / 2) {
      const int nzv = smode(kz, N);
      const int n2 = kx * kx + nyv * nyv + nzv * nzv;
      if (n2 > 0) {
        // |F_0|^2 = wc^2 a0, |F_2|^2 <= 5 wc^2 max(a0, a2/n^4), |F_4|^2 <= 155 wc^2 max(a0, a2/n^4, a4/n^8)
        // (triangle inequality on eqs. F2, delta4); the approximate reciprocal's
        // error is far inside the factor 2 of headroom in the scale below
        const float wc = wxy * zp.winv[2 * N + kz];
        float a = f0[i].x * f0[i].x + f0[i].y * f0[i].y;
        if (zp.lmax >= 2) {
          const float i2 = __fdividef(1.f, (float)n2), i4 = i2 * i2;
          a = fmaxf(a, (s2[i].x * s2[i].x + s2[i].y * s2[i].y) * i4);
          if (zp.lmax >= 4) a = fmaxf(a, (s4[i].x * s4[i].x + s4[i].y * s4[i].y) * i4 * i4);
        }
        float m = wc * wc * a * (zp.lmax >= 4 ? 155.f : (zp.lmax >= 2 ? 5.f : 1.f));
        if (MODE == 2 && n2 < zp.nsh2 && zp.slut[n2] >= 0) {
          const int w2 = 2 * zp.mm + 1;
          const size_t e = ((size_t)(nzv + zp.mm) * w2 + (nyv + zp.mm)) * (zp.mm + 1) + kx;
          const size_t es = (size_t)w2 * w2 * (zp.mm + 1);
          const float2 E0 = zp.E[e], E2 = zp.E[es + e], E4 = zp.E[2 * es + e];
          m = fmaxf(m, fmaxf(E0.x * E0.x + E0.y * E0.y, fmaxf(E2.x * E2.x + E2.y * E2.y, E4.x * E4.x + E4.y * E4.y)));
        }
        mloc = fmaxf(mloc, m);
      }
    }
  }
  {
    const unsigned mb = __reduce_max_sync(0xffffffffu, __float_as_uint(mloc));
    if ((threadIdx.x | (threadIdx.y & 3)) == 0) atomicMax(tmax, mb);  // lane 0 of each warp
  }
  __syncthreads();
  int et;
  frexpf(__uint_as_float(*tmax), &et);
  const int st = 49 - et;  // tile sum <= 2 * 8 N * M < 2^(13 + et) * 2^(49 - et) <= 2^62 (N <= 512)
  int curb = -1, cnt = 0;
  float acc[BQ_N];
#pragma unroll
  for (int q = 0; q < BQ_N; ++q) acc[q] = 0.f;
#pragma unroll
  for (int i = 0; i < PassShape<NT>::kRL; ++i) {
    const int kz = z0 + i;
    int b = -1;
    float vals[BQ_N];
#pragma unroll
    for (int q = 0; q < BQ_N; ++q) vals[q] = 0.f;
    if (colok && rowok && i < rl && kz < N && kz != N / 2) {
      const int nzv = smode(kz, N);
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
          if (nq > BQ_F42) {
            vals[BQ_F42] = F4.x * F2.x + F4.y * F2.y;
            vals[BQ_F44] = F4.x * F4.x + F4.y * F4.y;
          }
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
            // F0, F2, F4 are the Legendre fields of F^w here; E holds those of F
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
        for (int q = 0; q < BQ_N; ++q)
          if (q < nq)
            atomicAdd(reinterpret_cast<unsigned long long*>(sbi + q * nkey + curb),
                      (unsigned long long)__float2ll_rn(ldexpf(acc[q], q == BQ_K && MODE != 2 ? sk : st)));
      }
      curb = b;
      cnt = 0;
#pragma unroll
      for (int q = 0; q < BQ_N; ++q) acc[q] = 0.f;
    }
    if (b >= 0) {
      cnt += (int)wcol;
#pragma unroll
      for (int q = 0; q < BQ_N; ++q)
        if (q < nq) acc[q] = fmaf(wcol, vals[q], acc[q]);
    }
  }
  if (curb >= 0) {
    atomicAdd(sc + curb, cnt);
#pragma unroll
    for (int q = 0; q < BQ_N; ++q)
      if (q < nq)
        atomicAdd(reinterpret_cast<unsigned long long*>(sbi + q * nkey + curb),
                  (unsigned long long)__float2ll_rn(ldexpf(acc[q], q == BQ_K && MODE != 2 ? sk : st)));
  }
  __syncthreads();
  // the tile's fixed-point bin sums join the block's FP64 sums (each slot by
  // one thread, tiles in the block's order)
  for (int q = tid; q < BQ_N * nkey; q += NT) {
    sbd[q] += ldexp((double)sbi[q], (q / nkey == BQ_K && MODE != 2) ? -sk : -st);
    sbi[q] = 0;
  }
  if (tid == 0) *tmax = 0u;
  __syncthreads();
  }
  const int blk = blockIdx.x, nblk = gridDim.x;
  for (int q = tid; q < BQ_N * nkey; q += NT) part[(size_t)q * nblk + blk] = sbd[q];
  for (int q = tid; q < nkey; q += NT) partc[(size_t)q * nblk + blk] = sc[q];
}

// ----------------------------------------------------------------------------
// launch wrappers
// ----------------------------------------------------------------------------

int tiles_x(int N) { return (N / 2 + 1 + kT - 1) / kT; }

// The x-pass builds the moment fields from compile-time exponents; the host's
// moment table must list the fields in the same order.
bool moments_match(const MomentTable& mt) {
  for (int q = 0; q < mt.nfields; ++q)
    for (int a = 0; a < 3; ++a)
      if (mt.e[q][a] != field_exp(q, a)) return false;
  if (mt.ngroups > kMaxGroups) return false;
  for (int g = 0; g < mt.ngroups; ++g) {
    if (mt.g_f0[g] != zg_f0(g)) return false;
    // tables below ell = 2 (4) carry no S_2 (S_4) terms; the z-pass does not use them then
    if (mt.nfields >= nfields_of(2) && (mt.g_c2[g] != zg_c2(g) || (mt.g_c2[g] != 0.f && mt.g_p2[g] != zg_p2(g))))
      return false;
    if (mt.nfields == nfields_of(4) && (mt.g_c4[g] != zg_c4(g) || (mt.g_c4[g] != 0.f && mt.g_p4[g] != zg_p4(g))))
      return false;
  }
  return mt.nfields == nfields_of(4) || mt.nfields == nfields_of(2) || mt.nfields == nfields_of(0);
}
size_t field_elems(int N) { return (size_t)N * tiles_x(N) * N * kT; }
int yz_tiles(int N) { return tiles_x(N); }

static size_t xsm(int N, int NP) { return sizeof(float2) * (N + N / 2 + 2 * (size_t)NP * N); }
static size_t ysm(int N) { return 128 + sizeof(float2) * (3 * (size_t)N * kT + N); }
static size_t zsm(int N, int nkey) {
  return ysm(N) + sizeof(float2) * N + (sizeof(double) + sizeof(long long)) * BQ_N * nkey + sizeof(int) * nkey + 16;
}

// Persistent z-pass grid: one block per resident slot (two 256-thread or one
// 512-thread block per SM), at most one per tile.
int zpass_blocks(int N, int nt, int nsm) {
  const int ntiles = tiles_x(N) * N;
  const int nb = nsm * (nt == 256 ? 2 : 1);
  return nb < ntiles ? nb : ntiles;
}

template <int N_, int LMAX>
static cudaError_t xrun(const unsigned long long* gq, const float* gf, const GeomDev& g, const FftPlan& fp,
                        const float2* tw, float2* S1, int nsm, cudaStream_t s, int xm, const MockBatch& mb) {
  constexpr int NP = (nfields_of(LMAX) + 1) / 2;
  const size_t sm = xsm(g.N, NP);
  raise_smem_limit((const void*)k_xpass2<N_, LMAX>, sm);
  int occ = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_xpass2<N_, LMAX>, 32 * NP, sm);
  int grid = nsm * (occ > 0 ? occ : 1) * (xm > 0 ? xm : 2);
  if (grid > g.N * g.N) grid = g.N * g.N;
  k_xpass2<N_, LMAX><<<dim3(grid, 1, mb.n), dim3(NP, 32), sm, s>>>(gq, gf, g, fp, tw, S1, mb);
  return cudaGetLastError();
}

template <int LMAX>
static cudaError_t xdispatch(const unsigned long long* gq, const float* gf, const GeomDev& g, const FftPlan& fp,
                             const float2* tw, float2* S1, int nsm, cudaStream_t s, int xm, const MockBatch& mb) {
  if (LMAX == 4) {
    switch (g.N) {
      case 512: return xrun<512, LMAX>(gq, gf, g, fp, tw, S1, nsm, s, xm, mb);
      case 384: return xrun<384, LMAX>(gq, gf, g, fp, tw, S1, nsm, s, xm, mb);
      case 360: return xrun<360, LMAX>(gq, gf, g, fp, tw, S1, nsm, s, xm, mb);
      case 256: return xrun<256, LMAX>(gq, gf, g, fp, tw, S1, nsm, s, xm, mb);
      case 128: return xrun<128, LMAX>(gq, gf, g, fp, tw, S1, nsm, s, xm, mb);
      case 64: return xrun<64, LMAX>(gq, gf, g, fp, tw, S1, nsm, s, xm, mb);
      default: break;
    }
  }
  return xrun<0, LMAX>(gq, gf, g, fp, tw, S1, nsm, s, xm, mb);
}

cudaError_t launch_xpass(const unsigned long long* gq, const float* gf, const GeomDev& g, const MomentTable& mt,
                         const FftPlan& fp, const float2* tw, float2* S1, int nsm, cudaStream_t s, int xm,
                         MockBatch mb) {
  if (mt.nfields == nfields_of(4)) return xdispatch<4>(gq, gf, g, fp, tw, S1, nsm, s, xm, mb);
  if (mt.nfields == nfields_of(2)) return xdispatch<2>(gq, gf, g, fp, tw, S1, nsm, s, xm, mb);
  return xdispatch<0>(gq, gf, g, fp, tw, S1, nsm, s, xm, mb);
}

template <int N_, int NT>
static cudaError_t yrun_nt(const float2* S1, const unsigned long long* gq, const float* gf, const GeomDev& g,
                           const MomentTable& mt, const FftPlan& fp, const float2* tw, float2* S2, int* err,
                           cudaStream_t s, const MockBatch& mb) {
  const size_t sm = ysm(g.N);
  raise_smem_limit((const void*)k_ypass2<N_, NT>, sm);
  k_ypass2<N_, NT><<<dim3(tiles_x(g.N), g.N, mb.n), dim3(kT, NT / kT), sm, s>>>(S1, gq, gf, g, mt, fp, tw, S2, err,
                                                                                    mb);
  return cudaGetLastError();
}

template <int N_>
static cudaError_t yrun(const float2* S1, const unsigned long long* gq, const float* gf, const GeomDev& g,
                        const MomentTable& mt, const FftPlan& fp, const float2* tw, float2* S2, int* err,
                        cudaStream_t s, int nt, const MockBatch& mb) {
  return nt == 512 ? yrun_nt<N_, 512>(S1, gq, gf, g, mt, fp, tw, S2, err, s, mb)
                   : yrun_nt<N_, 256>(S1, gq, gf, g, mt, fp, tw, S2, err, s, mb);
}

// gq / gf: the grid the x-pass read (for the observer node's value).
cudaError_t launch_ypass(const float2* S1, const unsigned long long* gq, const float* gf, const GeomDev& g,
                         const MomentTable& mt, const FftPlan& fp, const float2* tw, float2* S2, int* err,
                         cudaStream_t s, int nt, MockBatch mb) {
  switch (g.N) {
    case 512: return yrun<512>(S1, gq, gf, g, mt, fp, tw, S2, err, s, nt, mb);
    case 384: return yrun<384>(S1, gq, gf, g, mt, fp, tw, S2, err, s, nt, mb);
    case 360: return yrun<360>(S1, gq, gf, g, mt, fp, tw, S2, err, s, nt, mb);
    case 256: return yrun<256>(S1, gq, gf, g, mt, fp, tw, S2, err, s, nt, mb);
    case 128: return yrun<128>(S1, gq, gf, g, mt, fp, tw, S2, err, s, nt, mb);
    case 64: return yrun<64>(S1, gq, gf, g, mt, fp, tw, S2, err, s, nt, mb);
    default: return yrun<0>(S1, gq, gf, g, mt, fp, tw, S2, err, s, nt, mb);
  }
}

template <int N_, int MODE, int NT>
static cudaError_t zrun_nt(const float2* S2, const GeomDev& g, const MomentTable& mt, const FftPlan& fp,
                           const float2* tw, const ZParams& zp, double* part, int* partc, int* err, cudaStream_t s,
                           int nsm, const MockBatch& mb) {
  const size_t sm = zsm(g.N, MODE == 2 ? zp.nshells : zp.nbins);
  raise_smem_limit((const void*)k_zpass2<N_, MODE, NT>, sm);
  k_zpass2<N_, MODE, NT><<<dim3(zpass_blocks(g.N, NT, nsm), 1, mb.n), dim3(kT, NT / kT), sm, s>>>(
      S2, g, mt, fp, tw, zp, part, partc, err, mb);
  return cudaGetLastError();
}

template <int N_, int MODE>
static cudaError_t zrun(const float2* S2, const GeomDev& g, const MomentTable& mt, const FftPlan& fp,
                        const float2* tw, const ZParams& zp, double* part, int* partc, int* err, cudaStream_t s,
                        int nsm, int nt, const MockBatch& mb) {
  return nt == 256 ? zrun_nt<N_, MODE, 256>(S2, g, mt, fp, tw, zp, part, partc, err, s, nsm, mb)
                   : zrun_nt<N_, MODE, 512>(S2, g, mt, fp, tw, zp, part, partc, err, s, nsm, mb);
}

template <int MODE>
static cudaError_t zdispatch(const float2* S2, const GeomDev& g, const MomentTable& mt, const FftPlan& fp,
                             const float2* tw, const ZParams& zp, double* part, int* partc, int* err,
                             cudaStream_t s, int nsm, int nt, const MockBatch& mb) {
  switch (g.N) {
    case 512: return zrun<512, MODE>(S2, g, mt, fp, tw, zp, part, partc, err, s, nsm, nt, mb);
    case 360: return zrun<360, MODE>(S2, g, mt, fp, tw, zp, part, partc, err, s, nsm, nt, mb);
    case 256: return zrun<256, MODE>(S2, g, mt, fp, tw, zp, part, partc, err, s, nsm, nt, mb);
    default: break;
  }
  if (MODE == 0) {
    switch (g.N) {
      case 384: return zrun<384, MODE>(S2, g, mt, fp, tw, zp, part, partc, err, s, nsm, nt, mb);
      case 128: return zrun<128, MODE>(S2, g, mt, fp, tw, zp, part, partc, err, s, nsm, nt, mb);
      case 64: return zrun<64, MODE>(S2, g, mt, fp, tw, zp, part, partc, err, s, nsm, nt, mb);
      default: break;
    }
  }
  return zrun<0, MODE>(S2, g, mt, fp, tw, zp, part, partc, err, s, nsm, nt, mb);
}

cudaError_t launch_zpass(const float2* S2, const GeomDev& g, const MomentTable& mt, const FftPlan& fp,
                         const float2* tw, const ZParams& zp, double* part, int* partc, int* err, cudaStream_t s,
                         int nsm, int nt, MockBatch mb) {
  if (zp.mode == 0) return zdispatch<0>(S2, g, mt, fp, tw, zp, part, partc, err, s, nsm, nt, mb);
  if (zp.mode == 1) return zdispatch<1>(S2, g, mt, fp, tw, zp, part, partc, err, s, nsm, nt, mb);
  return zdispatch<2>(S2, g, mt, fp, tw, zp, part, partc, err, s, nsm, nt, mb);
}

}  // namespace fkp
