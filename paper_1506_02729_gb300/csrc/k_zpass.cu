// k_zpass.cu - the z-pass of the power-spectrum path: FFT along z, Legendre
// recombination (eqs. F2, delta4), window compensation and shell binning (eq. shell)
// (shared helpers and layouts in k_fftpass.cuh).
#include "k_fftpass.cuh"

namespace fkp {

// One group's contribution to the thread's run of k_z: F_0 (F0), c2 nz^p2 to
// S_2 (A2), c4 nz^p4 to S_4 (A4).
template <int NZ, int RL, bool F0, bool A2, bool A4, bool PH>
__device__ __forceinline__ void zgroup(const float2* R, int z0, int rl, int N, int c, float c2, int p2, float c4,
                                       int p4, float2 (&f0)[RL], float2 (&s2)[RL], float2 (&s4)[RL],
                                       const float2* ph, float2 phxy) {
#pragma unroll
  for (int i = 0; i < RL; ++i) {
    const int kz = z0 + i;
    if (i < rl && kz < N) {
      float2 v = R[res_row<NZ, true>(kz) * kT + c];
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
  // one tile's fixed-point sums, [BQ_N][nkey] 64-bit integers held as low
  // words (sbl) and high words (sbh): 32-bit shared adds are native, a 64-bit
  // add is a compare-and-swap loop that contending threads repeat
  long long* sbi = reinterpret_cast<long long*>(sbd + BQ_N * nkey);
  unsigned* sbl = reinterpret_cast<unsigned*>(sbi);
  int* sbh = reinterpret_cast<int*>(sbl + BQ_N * nkey);
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
    const float2* R = fft_any<N_, kT, NT, -1, false, true>(bc, work, fp, tw);
    const int gg = gi < mt.ngroups ? gi : gi - mt.ngroups;  // the group's coefficients
    // second grid of an interlaced pair: its half-cell phase
    // e^{-i pi (n_x + n_y + n_z)/N}, the n_x, n_y part fixed per thread
    const float2 phxy = gi < mt.ngroups ? make_float2(1.f, 0.f)
                                        : cmul(zph[(t % NXT) * kT + c < N ? (t % NXT) * kT + c : 0], zph[t / NXT]);
    const int p2 = mt.g_p2[gg], p4 = mt.g_p4[gg];
    const float c2 = mt.g_c2[gg], c4 = mt.g_c4[gg];
    constexpr int RLc = PassShape<NT>::kRL;
    if (gi < mt.ngroups) {
      if (mt.g_f0[gg]) zgroup<N_, RLc, true, true, false, false>(R, z0, rl, N, c, c2, p2, c4, p4, f0, s2, s4, zph, phxy);
      else if (c2 != 0.f && c4 != 0.f) zgroup<N_, RLc, false, true, true, false>(R, z0, rl, N, c, c2, p2, c4, p4, f0, s2, s4, zph, phxy);
      else if (c2 != 0.f) zgroup<N_, RLc, false, true, false, false>(R, z0, rl, N, c, c2, p2, c4, p4, f0, s2, s4, zph, phxy);
      else zgroup<N_, RLc, false, false, true, false>(R, z0, rl, N, c, c2, p2, c4, p4, f0, s2, s4, zph, phxy);
    } else {  // second grid of an interlaced pair: its z half-cell phase
      if (mt.g_f0[gg]) zgroup<N_, RLc, true, true, false, true>(R, z0, rl, N, c, c2, p2, c4, p4, f0, s2, s4, zph, phxy);
      else if (c2 != 0.f && c4 != 0.f) zgroup<N_, RLc, false, true, true, true>(R, z0, rl, N, c, c2, p2, c4, p4, f0, s2, s4, zph, phxy);
      else if (c2 != 0.f) zgroup<N_, RLc, false, true, false, true>(R, z0, rl, N, c, c2, p2, c4, p4, f0, s2, s4, zph, phxy);
      else zgroup<N_, RLc, false, false, true, true>(R, z0, rl, N, c, c2, p2, c4, p4, f0, s2, s4, zph, phxy);
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
  // x added to slot j: the low word's carry out goes to the high word, so
  // sbh 2^32 + sbl is the exact sum (mod 2^64) whatever the order of adds
  auto add_fixed = [&](int j, long long x) {
    const unsigned lo = (unsigned)x;
    const unsigned old = atomicAdd(sbl + j, lo);
    atomicAdd(sbh + j, (int)(x >> 32) + (old + lo < old ? 1 : 0));
  };
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
            add_fixed(q * nkey + curb, __float2ll_rn(ldexpf(acc[q], q == BQ_K && MODE != 2 ? sk : st)));
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
        add_fixed(q * nkey + curb, __float2ll_rn(ldexpf(acc[q], q == BQ_K && MODE != 2 ? sk : st)));
  }
  __syncthreads();
  // the tile's fixed-point bin sums join the block's FP64 sums (each slot by
  // one thread, tiles in the block's order)
  for (int q = tid; q < BQ_N * nkey; q += NT) {
    const long long v = (long long)sbh[q] * 4294967296ll + (long long)sbl[q];
    sbd[q] += ldexp((double)v, (q / nkey == BQ_K && MODE != 2) ? -sk : -st);
    sbl[q] = 0u;
    sbh[q] = 0;
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
