// k_assign.cu - scalars and gridding of galaxies and randoms (Sec. III.A).
//
// Interpolation of the objects to the grid nodes (eq. mapFFT) with CIC, TSC or
// PCS (the paper's fourth-order) weights, as a counting sort by 16^3-cell tile followed by accumulation in
// shared memory:
//   count    per object: FKP weight and the partial sums of the scalars (W,
//            sum w^2, sum w^3, sum nbar w^2, sum nbar^2 w^3, for alpha, I_22,
//            I_33, N_0, S_3: eqs. I22def, N0true, Noise0) in double-single
//            arithmetic per thread and FP64 across threads,
//            the geometry check and one count for the object's tile (block
//            histogram in shared memory);
//   scan     tile offsets (exclusive prefix sum);
//   scatter  each object's (x, y, z, value) to its tile's segment, value =
//            w for galaxies and -alpha w for randoms (and the w^2-weighted
//            value for F^w, eq. SNbisp2), with the L^ab sums (eq. Lab);
//   tiles    one block per tile: every tap is rounded once to a 2^-40
//            fixed-point integer and added in shared memory over the tile and
//            its one-cell halo, then the nonzero cells are added to the grid.
// Integer sums make the grid independent of the order of the objects and of
// the blocks (deterministic, identical alone or inside a batch).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "fkp_internal.h"

namespace fkp {

constexpr int kTile = 16;            // cells per tile side
// Objects per work item of the tile accumulation: a tile's objects are split
// into items of at most this many, so that the few tiles of the densest
// parts of a survey do not hold up the end of the launch.
constexpr int kAccumChunk = 8160;
constexpr int kAccumThreads = 512;
// Region a tile's objects reach, from one cell below the tile: the tile
// plus one halo cell on each side for CIC and TSC, and one more above for
// PCS (taps c-1 .. c+2 of the centre cell c).
template <int P>
__host__ __device__ constexpr int reg_side() { return P == 4 ? kTile + 3 : kTile + 2; }
template <int P>
__host__ __device__ constexpr int reg_cells() { return reg_side<P>() * reg_side<P>() * reg_side<P>(); }

int assign_tiles_per_axis(int N) { return (N + kTile - 1) / kTile; }

// Centre cell of an object: TSC taps c-1..c+1 around c = floor(u + 1/2);
// CIC taps c, c+1 with c = floor(u); PCS taps c-1..c+2 with c = floor(u).
// Returns false when a tap would leave [1, N-2] (non-periodic) or the
// position is not finite.
template <int P>
__device__ __forceinline__ bool centre_cell(const GeomDev& g, float px, float py, float pz, int& cx, int& cy,
                                            int& cz) {
  const float ux = (px - g.ox) * g.invH, uy = (py - g.oy) * g.invH, uz = (pz - g.oz) * g.invH;
  const float sh = P == 3 ? 0.5f : 0.f;
  const int N = g.N;
  if (!g.periodic) {
    if (!(ux >= 0.f && ux < (float)N && uy >= 0.f && uy < (float)N && uz >= 0.f && uz < (float)N)) return false;
    cx = (int)floorf(ux + sh);
    cy = (int)floorf(uy + sh);
    cz = (int)floorf(uz + sh);
    const int lo = P == 2 ? 1 : 2, hi = P == 4 ? N - 4 : N - 3;
    return cx >= lo && cy >= lo && cz >= lo && cx <= hi && cy <= hi && cz <= hi;
  }
  if (!(fabsf(ux) < 1e8f && fabsf(uy) < 1e8f && fabsf(uz) < 1e8f)) return false;
  cx = (int)floorf(ux + sh);
  cy = (int)floorf(uy + sh);
  cz = (int)floorf(uz + sh);
  return true;
}

// i mod N in [0, N): indices within one box of the grid (all but periodic
// positions several boxes away) take the compare-and-add path, not a division.
__device__ __forceinline__ int wrapN(int i, int N) {
  if (i >= 0 && i < N) return i;
  if (i < 0 && i >= -N) return i + N;
  if (i >= N && i < 2 * N) return i - N;
  i %= N;
  return i < 0 ? i + N : i;
}

__device__ __forceinline__ int tile_of(int cx, int cy, int cz, int N, int ntx) {
  return ((wrapN(cz, N) / kTile) * ntx + wrapN(cy, N) / kTile) * ntx + wrapN(cx, N) / kTile;
}

// ---------------------------------------------------------------------------

// Each block owns a contiguous chunk of objects (the same chunks as the
// scatter launch on the same catalog): its counts go to a shared-memory
// histogram over all tiles, written out whole as the block's row of bh.
constexpr int kBinThreads = 1024;

template <int P>
__global__ void __launch_bounds__(kBinThreads) k_bin_count(CatDev c, int is_ran, GeomDev g, int ntx, int ntiles,
                                                           double* __restrict__ part, int* __restrict__ bh,
                                                           int* __restrict__ err) {
  extern __shared__ int hist[];
  __shared__ double sh[32];
  for (int t = threadIdx.x; t < ntiles; t += blockDim.x) hist[t] = 0;
  __syncthreads();
  FFSum s_w, s_w2, s_w3, s_nw2, s_n2w3;
  bool bad = false;
  const long long chunk = (c.n + gridDim.x - 1) / gridDim.x;
  const long long i0 = blockIdx.x * chunk;
  const long long i1 = i0 + chunk < c.n ? i0 + chunk : c.n;
  // unrolled: the loads of several objects in flight at once
#pragma unroll 4
  for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const FF w = fkp_weight_ff(c, i, g.P_fkp, g.P_fkp_lo);
    const FF w2 = ff_mul(w, w);
    const FF w3 = ff_mul(w2, w);
    s_w.add(w);
    s_w2.add(w2);
    s_w3.add(w3);
    if (is_ran) {
      const float nb = __ldg(c.nbar + i);
      const FF nw2 = ff_mul(w2, nb);
      s_nw2.add(nw2);
      s_n2w3.add(ff_mul(ff_mul(w3, nb), nb));
    }
    int cx, cy, cz;
    if (centre_cell<P>(g, __ldg(c.x + i), __ldg(c.y + i), __ldg(c.z + i), cx, cy, cz))
      atomicAdd(hist + tile_of(cx, cy, cz, g.N, ntx), 1);
    else
      bad = true;
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(err, 1);
  int* row = bh + (size_t)blockIdx.x * ntiles;
  for (int t = threadIdx.x; t < ntiles; t += blockDim.x) row[t] = hist[t];
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

// Per tile t, over the rows of bh (one per block of the count launches,
// galaxies' blocks first): each row's entry becomes the exclusive prefix of
// the rows above it, and cnt[t] the tile's total.  Rows are read in batches
// of 16 independent loads.
__global__ void __launch_bounds__(256) k_tile_prefix(int* __restrict__ bh, int nrows, int ntiles,
                                                     int* __restrict__ cnt) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntiles) return;
  int run = 0;
  for (int r0 = 0; r0 < nrows; r0 += 16) {
    int v[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = r0 + q < nrows ? bh[(size_t)(r0 + q) * ntiles + t] : 0;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      if (r0 + q < nrows) bh[(size_t)(r0 + q) * ntiles + t] = run;
      run += v[q];
    }
  }
  cnt[t] = run;
}

// Exclusive scan of the tile counts into offsets (off[ntiles] = total), and
// of the tiles' work items (one per
// kAccumChunk objects or part of it) into item offsets (items[ntiles] = the
// number of items).  One block of 1024 threads walks the tiles in rounds of
// 1024 (coalesced loads, the next round's counts loaded during this round's
// warp-shuffle scan).
__global__ void __launch_bounds__(1024) k_scan_tiles(const int* __restrict__ cnt, int ntiles, int* __restrict__ off,
                                                     int* __restrict__ items) {
  __shared__ int wsum[32], wsumi[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int carry = 0, carryi = 0;  // totals of the earlier rounds (the same in every thread)
  int c = (int)threadIdx.x < ntiles ? cnt[threadIdx.x] : 0;
  for (int base = 0; base < ntiles; base += 1024) {
    const int i = base + (int)threadIdx.x;
    const int cn = i + 1024 < ntiles ? cnt[i + 1024] : 0;
    const int ci = (c + kAccumChunk - 1) / kAccumChunk;
    int s = c, si = ci;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, s, o), vi = __shfl_up_sync(0xffffffffu, si, o);
      if (lane >= o) {
        s += v;
        si += vi;
      }
    }
    if (lane == 31) {
      wsum[warp] = s;
      wsumi[warp] = si;
    }
    __syncthreads();
    if (warp == 0) {
      int w = wsum[lane], wi = wsumi[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, w, o), vi = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= o) {
          w += v;
          wi += vi;
        }
      }
      wsum[lane] = w;
      wsumi[lane] = wi;
    }
    __syncthreads();
    if (i < ntiles) {
      const int e = carry + (warp ? wsum[warp - 1] : 0) + s - c;
      off[i] = e;
      items[i] = carryi + (warp ? wsumi[warp - 1] : 0) + si - ci;
    }
    carry += wsum[31];
    carryi += wsumi[31];
    __syncthreads();
    c = cn;
  }
  if (threadIdx.x == 0) {
    off[ntiles] = carry;
    items[ntiles] = carryi;
  }
}

// Each block owns the contiguous chunk of objects its count block counted:
// its range inside tile t's segment starts at off[t] plus the counts of the
// blocks before it (its row of the prefixed bh), so one pass over the chunk
// writes each object at the next slot of its tile's range.
// raw = 1 (randoms only): values w and w^2 without alpha, for the cached
// random grids that later mocks combine with their own alpha.
template <int P>
__global__ void __launch_bounds__(kBinThreads) k_bin_scatter(CatDev c, int is_ran, int raw, GeomDev g, int ntx,
                                                             int ntiles, float obx, float oby, float obz,
                                                             const double* __restrict__ ds,
                                                             const int* __restrict__ off,
                                                             const int* __restrict__ bpref,
                                                             float4* __restrict__ xyzv, float* __restrict__ vw2,
                                                             double* __restrict__ labpart) {
  extern __shared__ int hist[];
  __shared__ double sh[32];
  // alpha and alpha^2 as float pairs (hi + lo): each random's value is then
  // rounded once, at random, instead of carrying the FP32 rounding of alpha
  // into every random alike (a systematic scale of the random field)
  const double ad = raw ? 0.0 : ds[DS_ALPHA];
  const float alpha = (float)ad, alo = (float)(ad - (double)alpha);
  const float a2 = (float)(ad * ad), a2lo = (float)(ad * ad - (double)a2);
  const long long chunk = (c.n + gridDim.x - 1) / gridDim.x;
  const long long i0 = blockIdx.x * chunk;
  const long long i1 = i0 + chunk < c.n ? i0 + chunk : c.n;
  const int* brow = bpref + (size_t)blockIdx.x * ntiles;
  for (int t = threadIdx.x; t < ntiles; t += blockDim.x) hist[t] = off[t] + brow[t];
  __syncthreads();
  KahanF lab[LAB_NSUM];
  // unrolled: the loads of several objects in flight at once
#pragma unroll 4
  for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const float w = fkp_weight(c, i, g.P_fkp);
    const float px = __ldg(c.x + i), py = __ldg(c.y + i), pz = __ldg(c.z + i);
    int cx, cy, cz;
    if (centre_cell<P>(g, px, py, pz, cx, cy, cz)) {
      const int slot = atomicAdd(hist + tile_of(cx, cy, cz, g.N, ntx), 1);
      xyzv[slot] = make_float4(px, py, pz, is_ran && !raw ? -fmaf(alpha, w, alo * w) : w);
      if (vw2) {
        const float ww = w * w;
        vw2[slot] = is_ran && !raw ? fmaf(a2, ww, a2lo * ww) : ww;
      }
    }
    if (is_ran) {
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
  if (is_ran) {
#pragma unroll
    for (int q = 0; q < LAB_NSUM; ++q) {
      const double v = block_sum_f64(lab[q].value(), sh);
      if (threadIdx.x == 0) labpart[(size_t)blockIdx.x * LAB_NSUM + q] = v;
    }
  }
}

template <int P>
__device__ __forceinline__ void tap_weights(float u, int& i0, float* wt) {
  if (P == 2) {
    const float f = floorf(u);
    const float d = u - f;
    i0 = (int)f;
    wt[0] = 1.f - d;
    wt[1] = d;
  } else if (P == 3) {
    const float f = floorf(u + 0.5f);
    const float d = u - f;
    i0 = (int)f - 1;
    const float a = 0.5f - d, b = 0.5f + d;
    wt[0] = 0.5f * a * a;
    wt[1] = 0.75f - d * d;
    wt[2] = 0.5f * b * b;
  } else {
    // PCS: the cubic B-spline at distances 1 + d, d, 1 - d, 2 - d
    const float f = floorf(u);
    const float d = u - f;
    i0 = (int)f - 1;
    const float e = 1.f - d, d2 = d * d, d3 = d2 * d;
    wt[0] = e * e * e * (1.f / 6.f);
    wt[1] = (4.f - 6.f * d2 + 3.f * d3) * (1.f / 6.f);
    wt[2] = (1.f + 3.f * (d + d2 - d3)) * (1.f / 6.f);
    wt[3] = d3 * (1.f / 6.f);
  }
}

// x = round(v 2^40) as h 2^19 + l with FP32 arithmetic only (no conversion
// instructions): for |v| < 2, adding M = 1.5 2^23 to v 2^21 (one FMA, one
// rounding to nearest even) leaves h = round(v 2^21) in the low bits of the
// sum; the remainder v 2^21 - h is exact and lies in [-1/2, 1/2], and a
// second FMA leaves l = round((v 2^21 - h) 2^19) in [-2^18, 2^18] the same
// way.  h 2^19 + l is round(v 2^40), rounded to nearest even, exactly.
constexpr float kMagic = 12582912.0f;   // 1.5 2^23
constexpr int kMagicBits = 0x4B400000;  // its bit pattern
__device__ __forceinline__ void split_fixed(float v, int& h, int& l) {
  const float a = fmaf(v, 2097152.0f, kMagic);  // v 2^21 + M
  const float hf = a - kMagic;
  const float rem = fmaf(v, 2097152.0f, -hf);
  h = __float_as_int(a) - kMagicBits;
  l = __float_as_int(fmaf(rem, 524288.0f, kMagic)) - kMagicBits;
}

// x^_x^ea x^_y^eb x^_z^ec of the object at (o.x, o.y, o.z): its own line of
// sight about the observer (node 0 sits at origin - observer = (rx, ry, rz)
// from it), the fixed one for an observer at infinity; x^ = 0 at the
// observer itself.
__device__ __forceinline__ float ipow(float v, int e) {
  float r = 1.f;
  for (int k = 0; k < e; ++k) r *= v;
  return r;
}
__device__ __forceinline__ float object_moment(const GeomDev& g, const float4& o, int ea, int eb, int ec) {
  float hx = g.lx, hy = g.ly, hz = g.lz;
  if (!g.los_inf) {
    const float dx = (o.x - g.ox) + g.rx, dy = (o.y - g.oy) + g.ry, dz = (o.z - g.oz) + g.rz;
    const float r2 = dx * dx + dy * dy + dz * dz;
    const float inv = r2 > 0.f ? rsqrtf(r2) : 0.f;
    hx = dx * inv;
    hy = dy * inv;
    hz = dz * inv;
  }
  return ipow(hx, ea) * ipow(hy, eb) * ipow(hz, ec);
}

// One block per work item: up to kAccumChunk objects of one tile (items in
// tile order; items[t] is tile t's first).  The tile's region, from one cell
// below the tile to the end of its reach (reg_side cells a side), covers the
// taps of every object whose centre cell lies in the tile.  Blocks past the
// last item return at once (the grid is sized from an upper bound).
//
// Each tap adds x = round(v 2^40) to its cell (v = w times the tap weight).
// Shared-memory adds of 64 bits are several times slower than adds of 32
// bits, and conversions to 64-bit integers run on a narrow pipe, so when the
// item allows it a cell is held as two signed 32-bit words from split_fixed:
// L sums the l (at most kAccumChunk < 2^13 terms of magnitude <= 2^18: |L| <
// 2^31) and H the h.  H stays exact while the item's sum S of |w| (an upper
// bound for any cell's sum of |v|, every tap weight being at most 1) is
// below 2^10 - 1: then |H| <= 2^21 S + 2^12 < 2^31.  split_fixed needs |v| <
// 2.  Items that fail either bound add x = round(v 2^40) as one 64-bit word
// instead.  Both forms give the exact integer sum of the x, so the grid does
// not depend on how the objects are split into items or in which order they
// are added.
template <int P, bool W2>
__global__ void __launch_bounds__(kAccumThreads, W2 ? 2 : 4) k_tile_accum(GeomDev g, int ntx, int ntiles,
                                                                        const int* __restrict__ off,
                                                                        const int* __restrict__ items,
                                                                        const float4* __restrict__ xyzv,
                                                                        const float* __restrict__ vw2,
                                                                        unsigned long long* __restrict__ grid,
                                                                        unsigned long long* __restrict__ gridw,
                                                                        int ea, int eb, int ec) {
  constexpr int kReg = reg_side<P>(), kReg3 = reg_cells<P>();
  static_assert(kAccumChunk * 262144ll < 2147483648ll, "the low words would wrap");
  extern __shared__ unsigned long long reg[];
  __shared__ int s_tile;
  __shared__ float s_abs;
  __shared__ int s_max;
  unsigned long long* regw = reg + kReg3;
  int* L = reinterpret_cast<int*>(reg);
  int* H = L + kReg3;
  int* Lw = reinterpret_cast<int*>(regw);
  int* Hw = Lw + kReg3;
  const int item = blockIdx.x;
  if (item >= items[ntiles]) return;
  if (threadIdx.x == 0) {
    // last tile whose first item is at or before this one
    int lo = 0, hi = ntiles - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (items[mid] <= item) lo = mid;
      else hi = mid - 1;
    }
    s_tile = lo;
    s_abs = 0.f;
    s_max = 0;
  }
  const int N = g.N;
  for (int i = threadIdx.x; i < kReg3; i += blockDim.x) {
    reg[i] = 0ull;
    if (W2) regw[i] = 0ull;
  }
  __syncthreads();
  const int t = s_tile;
  const int a = off[t] + (item - items[t]) * kAccumChunk;
  const int b = min(off[t + 1], a + kAccumChunk);
  const int tx = t % ntx, ty = (t / ntx) % ntx, tz = t / (ntx * ntx);
  const int lx0 = tx * kTile - 1, ly0 = ty * kTile - 1, lz0 = tz * kTile - 1;
  // the item's objects are read twice: for the bounds, then for the taps
  float sa = 0.f, ma = 0.f;
  for (int i = a + threadIdx.x; i < b; i += kAccumThreads) {
    const float m = fmaxf(fabsf(xyzv[i].w), W2 ? fabsf(vw2[i]) : 0.f);
    sa += m;
    ma = fmaxf(ma, m);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sa += __shfl_xor_sync(0xffffffffu, sa, o);
    ma = fmaxf(ma, __shfl_xor_sync(0xffffffffu, ma, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&s_abs, sa);
    atomicMax(&s_max, __float_as_int(ma));  // non-negative: ordered as integers (NaN above +inf)
  }
  __syncthreads();
  // the bounds, with room for the rounding of the FP32 sums above
  const bool split = s_abs < 1000.f && __int_as_float(s_max) < 2.f;
  for (int i = a + threadIdx.x; i < b; i += kAccumThreads) {
    float4 o = xyzv[i];
    const float wv = W2 ? vw2[i] : 0.f;
    if (ea >= 0) o.w *= object_moment(g, o, ea, eb, ec);  // |x^ products| <= 1: the bounds hold
    const float ux = (o.x - g.ox) * g.invH, uy = (o.y - g.oy) * g.invH, uz = (o.z - g.oz) * g.invH;
    int ix, iy, iz;
    float wx[P], wy[P], wz[P];
    tap_weights<P>(ux, ix, wx);
    tap_weights<P>(uy, iy, wy);
    tap_weights<P>(uz, iz, wz);
    // taps relative to the region (periodic positions may lie one box away)
    const int cx = ix + (P >= 3 ? 1 : 0), cy = iy + (P >= 3 ? 1 : 0), cz = iz + (P >= 3 ? 1 : 0);
    const int rx = ix - (cx - wrapN(cx, N)) - lx0;
    const int ry = iy - (cy - wrapN(cy, N)) - ly0;
    const int rz = iz - (cz - wrapN(cz, N)) - lz0;
    if (split) {
#pragma unroll
      for (int p = 0; p < P; ++p) {
#pragma unroll
        for (int q = 0; q < P; ++q) {
          const float wzy = wz[p] * wy[q];
          const int base = ((rz + p) * kReg + (ry + q)) * kReg + rx;
#pragma unroll
          for (int r = 0; r < P; ++r) {
            const float tw = wzy * wx[r];
            int h, l;
            split_fixed(o.w * tw, h, l);
            atomicAdd(L + base + r, l);
            atomicAdd(H + base + r, h);
            if (W2) {
              split_fixed(wv * tw, h, l);
              atomicAdd(Lw + base + r, l);
              atomicAdd(Hw + base + r, h);
            }
          }
        }
      }
    } else {
#pragma unroll
      for (int p = 0; p < P; ++p) {
#pragma unroll
        for (int q = 0; q < P; ++q) {
          const float wzy = wz[p] * wy[q];
          const int base = ((rz + p) * kReg + (ry + q)) * kReg + rx;
#pragma unroll
          for (int r = 0; r < P; ++r) {
            const float tw = wzy * wx[r];
            atomicAdd(reg + base + r, (unsigned long long)__float2ll_rn(o.w * tw * kFixScaleF));
            if (W2) atomicAdd(regw + base + r, (unsigned long long)__float2ll_rn(wv * tw * kFixScaleF));
          }
        }
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kReg3; i += blockDim.x) {
    unsigned long long v, vw = 0ull;
    if (split) {
      v = (unsigned long long)((long long)H[i] * 524288ll + (long long)L[i]);
      if (W2) vw = (unsigned long long)((long long)Hw[i] * 524288ll + (long long)Lw[i]);
    } else {
      v = reg[i];
      if (W2) vw = regw[i];
    }
    if (v == 0ull && vw == 0ull) continue;
    const int lx = i % kReg, ly = (i / kReg) % kReg, lz = i / (kReg * kReg);
    const size_t gi = ((size_t)wrapN(lz0 + lz, N) * N + wrapN(ly0 + ly, N)) * N + wrapN(lx0 + lx, N);
    if (v) atomicAdd(grid + gi, v);
    if (W2 && vw) atomicAdd(gridw + gi, vw);
  }
}

// F = G - alpha R and F^w = G^w + alpha^2 R^w (eqs. mapFFT, SNbisp2) from the
// galaxies' fixed-point grids G, G^w and the cached random grids R = sum_r w W,
// R^w = sum_r w^2 W: each random term is rounded once to the grid's 2^-40
// fixed point, so the result is as deterministic as a direct gridding.
__global__ void __launch_bounds__(256) k_combine_randoms(unsigned long long* __restrict__ grid,
                                                         const unsigned long long* __restrict__ rgrid,
                                                         unsigned long long* __restrict__ gridw,
                                                         const unsigned long long* __restrict__ rgridw,
                                                         const double* __restrict__ ds, long long n) {
  const double a = ds[DS_ALPHA];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    grid[i] = (unsigned long long)((long long)grid[i] - __double2ll_rn(a * (double)(long long)__ldg(rgrid + i)));
    if (gridw)
      gridw[i] = (unsigned long long)((long long)gridw[i] +
                                      __double2ll_rn(a * a * (double)(long long)__ldg(rgridw + i)));
  }
}

// ---------------------------------------------------------------------------
// launch wrappers
// ---------------------------------------------------------------------------

cudaError_t launch_combine_randoms(unsigned long long* grid, const unsigned long long* rgrid,
                                   unsigned long long* gridw, const unsigned long long* rgridw, const double* ds,
                                   long long n, int nsm, cudaStream_t s) {
  long long nb = (n + 255) / 256;
  if (nb > (long long)nsm * 16) nb = (long long)nsm * 16;
  k_combine_randoms<<<(int)nb, 256, 0, s>>>(grid, rgrid, gridw, rgridw, ds, n);
  return cudaGetLastError();
}

// bh: the nblk rows (ntiles ints each) this launch fills.
cudaError_t launch_bin_count(const CatDev& c, int is_ran, const GeomDev& g, double* part, int* bh, int* err,
                             int nblk, cudaStream_t s) {
  const int ntx = assign_tiles_per_axis(g.N);
  const int ntiles = ntx * ntx * ntx;
  if (c.n == 0) {
    cudaMemsetAsync(part, 0, sizeof(double) * SC_NSUM * nblk, s);
    cudaMemsetAsync(bh, 0, sizeof(int) * (size_t)ntiles * nblk, s);
    return cudaGetLastError();
  }
  const size_t sm = sizeof(int) * ntiles;
  if (g.assign == 2) {
    raise_smem_limit((const void*)k_bin_count<2>, sm);
    k_bin_count<2><<<nblk, kBinThreads, sm, s>>>(c, is_ran, g, ntx, ntiles, part, bh, err);
  } else if (g.assign == 3) {
    raise_smem_limit((const void*)k_bin_count<3>, sm);
    k_bin_count<3><<<nblk, kBinThreads, sm, s>>>(c, is_ran, g, ntx, ntiles, part, bh, err);
  } else {
    raise_smem_limit((const void*)k_bin_count<4>, sm);
    k_bin_count<4><<<nblk, kBinThreads, sm, s>>>(c, is_ran, g, ntx, ntiles, part, bh, err);
  }
  return cudaGetLastError();
}

cudaError_t launch_tile_prefix(int* bh, int nrows, int ntiles, int* cnt, cudaStream_t s) {
  k_tile_prefix<<<(ntiles + 255) / 256, 256, 0, s>>>(bh, nrows, ntiles, cnt);
  return cudaGetLastError();
}

cudaError_t launch_scan_tiles(const int* cnt, int ntiles, int* off, int* items, cudaStream_t s) {
  k_scan_tiles<<<1, 1024, 0, s>>>(cnt, ntiles, off, items);
  return cudaGetLastError();
}

// off: the tile offsets; bpref: the nblk prefixed count rows of this catalog.
cudaError_t launch_bin_scatter(const CatDev& c, int is_ran, const GeomDev& g, const double obs[3], const double* ds,
                               const int* off, const int* bpref, float4* xyzv, float* vw2, double* labpart, int nblk,
                               cudaStream_t s, int raw) {
  if (c.n == 0) {
    if (is_ran) cudaMemsetAsync(labpart, 0, sizeof(double) * LAB_NSUM * nblk, s);
    return cudaGetLastError();
  }
  const int ntx = assign_tiles_per_axis(g.N);
  const int ntiles = ntx * ntx * ntx;
  const size_t sm = sizeof(int) * ntiles;
  if (g.assign == 2) {
    raise_smem_limit((const void*)k_bin_scatter<2>, sm);
    k_bin_scatter<2><<<nblk, kBinThreads, sm, s>>>(c, is_ran, raw, g, ntx, ntiles, (float)obs[0], (float)obs[1],
                                                   (float)obs[2], ds, off, bpref, xyzv, vw2, labpart);
  } else if (g.assign == 3) {
    raise_smem_limit((const void*)k_bin_scatter<3>, sm);
    k_bin_scatter<3><<<nblk, kBinThreads, sm, s>>>(c, is_ran, raw, g, ntx, ntiles, (float)obs[0], (float)obs[1],
                                                   (float)obs[2], ds, off, bpref, xyzv, vw2, labpart);
  } else {
    raise_smem_limit((const void*)k_bin_scatter<4>, sm);
    k_bin_scatter<4><<<nblk, kBinThreads, sm, s>>>(c, is_ran, raw, g, ntx, ntiles, (float)obs[0], (float)obs[1],
                                                   (float)obs[2], ds, off, bpref, xyzv, vw2, labpart);
  }
  return cudaGetLastError();
}

// nobj: the objects scattered into tile order (bounds the number of items).
cudaError_t launch_tile_accum(const GeomDev& g, const int* off, const int* items, long long nobj, const float4* xyzv,
                              const float* vw2, unsigned long long* grid, unsigned long long* gridw, cudaStream_t s,
                              const unsigned char* xe) {
  const int ea = xe ? xe[0] : -1, eb = xe ? xe[1] : 0, ec = xe ? xe[2] : 0;
  const int ntx = assign_tiles_per_axis(g.N);
  const int ntiles = ntx * ntx * ntx;
  // every non-empty tile has one item that may be partial, the rest are full
  const long long nitems = std::min<long long>((long long)ntiles, nobj) + nobj / kAccumChunk;
  if (nitems <= 0) return cudaSuccess;
  if (nitems > INT32_MAX) return cudaErrorInvalidValue;
  const bool w2 = gridw != nullptr;
#define FKP_TA(PP, WW)                                                                                 \
  do {                                                                                                 \
    const size_t sm = sizeof(unsigned long long) * reg_cells<PP>() * (WW ? 2 : 1);                     \
    raise_smem_limit((const void*)k_tile_accum<PP, WW>, sm);                                           \
    k_tile_accum<PP, WW><<<(int)nitems, kAccumThreads, sm, s>>>(g, ntx, ntiles, off, items, xyzv, vw2, grid, \
                                                                gridw, ea, eb, ec);                    \
  } while (0)
  if (g.assign == 2) {
    if (w2) FKP_TA(2, true); else FKP_TA(2, false);
  } else if (g.assign == 3) {
    if (w2) FKP_TA(3, true); else FKP_TA(3, false);
  } else {
    if (w2) FKP_TA(4, true); else FKP_TA(4, false);
  }
#undef FKP_TA
  return cudaGetLastError();
}

}  // namespace fkp
