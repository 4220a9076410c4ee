// k_contract_tc.cu - the triangle contraction of eq. Factorize on the
// tcgen05 tensor cores.
//
//   T^(l)(a,b,c) = sum_x F_a^(l)(x) F_b^(0)(x) F_c^(0)(x)
//
// is the skinny GEMM D[(l,a), (b,c)] = sum_x A[(l,a), x] B[(b,c), x] with
// A = the shell fields and B = the Khatri-Rao products F_b^(0) F_c^(0).  Each
// FP32 operand v is split into BF16 v_hi = bf16(v), v_lo = bf16(v - v_hi); the
// three products hi*hi + hi*lo + lo*hi are accumulated in FP32 in tensor
// memory (the lo*lo term and the rounding of lo, each ~2^-18 relative, are
// dropped: a per-product error of random sign, which over N^3 points
// random-walks to ~2^-17 sqrt(sum_x t^2) on a triangle sum).  The 3-way
// split v = v_hi + v_mid + v_lo keeps the six products whose order is at most
// 2^-16 (hh, hm, mh, hl, lh, mm), for a per-term error near FP32 rounding:
// the triangle sums cancel strongly (sum |t| >> |sum t|), so the 3-way split
// is the accurate mode and the 2-way split the fast one.
//
// One CTA of 16 warps per (256-column N tile, K slice).  The slices (up to
// about 4,096 chunks of 32 points) are sized at plan time so that tiles x
// slices CTAs fill whole waves of the SMs.
// The shell fields of a chunk of 32 points are fetched two chunks ahead with
// cp.async into a 3-slot ring; operand stages are double buffered: all
// threads form the products and the BF16 splits into K-major tiles with the
// 64-byte swizzle (one 64-byte row of K per operand row); one thread issues
// the tcgen05.mma instructions (M = 128, N = 256, K = 16) and commits them to
// the stage's mbarrier.  After every run of 96 accumulating MMAs (16 chunks,
// 8 for the 3-way split) the 128 x 256 FP32 tile is read from tensor memory
// (tcgen05.ld; each warp its lane quarter and 64 columns), added with
// round-to-nearest to a running FP32 sum held in the other 256 tensor-memory
// columns (tcgen05.ld, add, tcgen05.st) and the MMA accumulation restarts.
// In-tensor-core accumulation runs were measured to drift linearly with their
// length (5.6e-4 of the monopole scale over 65,536 points, under 1e-4 over
// 1,024).  With 1,024-point runs that rounding, not the operand split, set
// the 3-way split's error (B_4 8.4e-5 of the FP32 contraction on a 64^3
// case, above the 2-way split's 5.1e-5); with runs of 96 MMAs it is 6.7e-6.
// The drain of a run waits until the next chunk's operands are built, so the
// tensor pipe idles only for the drain.  At the end of the slice the sums go
// to per-slice partials, summed over slices in FP64 by k_tc_reduce.
#include <algorithm>

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fkp_internal.h"

namespace fkp {

constexpr int kTcM = 128;              // MMA rows (l, a)
constexpr int kTcN = 256;              // MMA columns (pairs b >= c) per tile
constexpr int kTcKC = 32;              // K points per chunk
constexpr int kTcSliceTarget = 4096;   // chunks per K slice, at most (about)
constexpr int kTcThreads = 512;
constexpr int kTcABytes = kTcM * kTcKC * 2;    // one BF16 operand tile: 8 KB
constexpr int kTcBBytes = kTcN * kTcKC * 2;    // 16 KB
template <int NS>
__host__ __device__ constexpr int tc_stage_bytes() { return NS * (kTcABytes + kTcBBytes); }
constexpr int kTcRow = kTcKC + 4;      // staged row stride (floats): 16-byte aligned, shifts banks by 4 per field

// chunks per tensor-memory accumulation run: 96 accumulating MMAs per run for
// every split (3 products x 2 K steps x 16 chunks; 6 x 2 x 8)
template <int NS>
__host__ __device__ constexpr int tc_drain() { return NS == 3 ? 8 : 16; }
// K slicing: the fewest whole waves of the SMs (tiles x slices CTAs, one per
// SM at a time) whose slices hold at most about kTcSliceTarget chunks; slices
// of equal length (the last one shorter), none empty.
void tc_slicing(long long N3, int ntiles, int nsm, int* nslices, int* chunks) {
  const long long total = (N3 + kTcKC - 1) / kTcKC;
  const long long per_wave = (long long)nsm * kTcSliceTarget;
  const long long waves = std::max<long long>(1, (total * ntiles + per_wave - 1) / per_wave);
  long long ns = std::max<long long>(1, waves * nsm / std::max(1, ntiles));
  ns = std::min(ns, std::max<long long>(1, total));
  const long long ch = (total + ns - 1) / ns;
  *chunks = (int)ch;
  *nslices = (int)((total + ch - 1) / ch);
}
int tc_tile_cols() { return kTcN; }
int tc_rows() { return kTcM; }

// ---------------------------------------------------------------------------
// tcgen05 / TMEM wrappers
// ---------------------------------------------------------------------------

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A * B^T, A and B K-major BF16 in shared memory, FP32 accumulate.
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 32 consecutive FP32 columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 32 consecutive FP32 columns of this warp's 32 TMEM lanes, stored.
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const float* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};"
      ::"r"(taddr), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
        "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
        "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
        "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
        "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
        "r"(__float_as_uint(v[15])), "r"(__float_as_uint(v[16])), "r"(__float_as_uint(v[17])),
        "r"(__float_as_uint(v[18])), "r"(__float_as_uint(v[19])), "r"(__float_as_uint(v[20])),
        "r"(__float_as_uint(v[21])), "r"(__float_as_uint(v[22])), "r"(__float_as_uint(v[23])),
        "r"(__float_as_uint(v[24])), "r"(__float_as_uint(v[25])), "r"(__float_as_uint(v[26])),
        "r"(__float_as_uint(v[27])), "r"(__float_as_uint(v[28])), "r"(__float_as_uint(v[29])),
        "r"(__float_as_uint(v[30])), "r"(__float_as_uint(v[31]))
      : "memory");
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// tcgen05.ld of 32 columns without the wait, and the wait that completes
// every load in flight; the wait names the destination registers as in-out
// operands so that no use of them is moved ahead of it.
__device__ __forceinline__ void tmem_ld32_async(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_wait_ld(uint32_t* r) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                 "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                 "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                 "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
               :
               : "memory");
}
// tcgen05.st of 32 columns without the wait (tcgen05.wait::st completes it)
__device__ __forceinline__ void tmem_st32_async(uint32_t taddr, const uint32_t* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};"
      ::"r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
        "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]),
        "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]),
        "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand with the 64-byte swizzle.
// Each row holds the chunk's 32 K values (64 bytes); 8 rows form a 512-byte
// swizzle atom (sbo = 512 between atoms); the K steps of 16 advance the start
// address by 32 bytes within the rows.  Descriptor version 1, layout type
// SWIZZLE_64B (4) in bits 61-63.
__device__ __forceinline__ uint64_t sdesc(const void* p, uint32_t lbo, uint32_t sbo) {
  const uint64_t a = (uint64_t)((smem_u32(p) & 0x3FFFF) >> 4);
  return a | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) | (1ull << 46) | (4ull << 61);
}

// Instruction descriptor for kind::f16: D FP32, A and B BF16, both K-major,
// N = 256, M = 128.
__host__ __device__ constexpr uint32_t tc_idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcN >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
}

// Byte offset of the 16-byte segment (row, k-group kg) of an operand tile in
// the 64-byte-swizzled K-major layout: row r at 64 r, its 16-byte chunk kg
// stored at chunk kg ^ ((r >> 1) & 3) (address bits 4-5 XOR bits 7-8).  A
// quarter-warp storing 8 consecutive rows of one kg hits 8 distinct 16-byte
// bank groups.
__device__ __forceinline__ int canon_off(int row, int kg) {
  return row * 64 + ((kg ^ ((row >> 1) & 3)) << 4);
}

// BF16 split of 8 values into NS parts (each part the BF16 rounding of the
// remainder), packed 16 bytes per part.
template <int NS>
__device__ __forceinline__ void split8(const float* v, uint4* out) {
  uint32_t w[NS][4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float2 r = make_float2(v[2 * i], v[2 * i + 1]);
#pragma unroll
    for (int p = 0; p < NS; ++p) {
      const __nv_bfloat162 h = __floats2bfloat162_rn(r.x, r.y);  // one paired conversion
      w[p][i] = *reinterpret_cast<const uint32_t*>(&h);
      if (p + 1 < NS) {
        const float2 hf = __bfloat1622float2(h);
        r.x -= hf.x;
        r.y -= hf.y;
      }
    }
  }
#pragma unroll
  for (int p = 0; p < NS; ++p) out[p] = make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
}

// ---------------------------------------------------------------------------

// pairs: (b, c) of the tile's columns (b < 0 marks padding); part layout
// [slice][tile][128][256] FP32.
//
// Every thread has a fixed share of each chunk: A row t % 128, k-group t / 128
// (8 points); B row t % 256, k-groups 2 (t / 256) and 2 (t / 256) + 1 (16
// points); its field copies are f = i / 8, points 4 (i % 8) of i = t, t + 512.
// Offsets and pair indices are therefore computed once.  Rows of A beyond nf
// and padding columns of B are zeroed once in both stages and never
// rewritten.  The running FP32 sum of the drained tiles sits in tensor memory
// columns 256-511 (each drain: tcgen05.ld tile and sum, add, tcgen05.st), so
// no accumulator occupies registers through the chunk loop.
template <int NS>
__global__ void __launch_bounds__(kTcThreads, 1) k_contract_tc(const float* __restrict__ I, long long N3, int nf,
                                                               int S, const short2* __restrict__ pairs, int npairs,
                                                               int chunks, float* __restrict__ part,
                                                               int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  constexpr int kStage = tc_stage_bytes<NS>();
  unsigned char* stage0 = smraw;                                  // 2 stages: A parts, then B parts
  float* Iring = reinterpret_cast<float*>(smraw + 2 * kStage);   // 3 x [nf][kTcRow], prefetched 2 chunks ahead
  const int ring = nf * kTcRow;                                   // floats per ring slot
  uint64_t* bar = reinterpret_cast<uint64_t*>(Iring + 3 * ring);  // [2]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int tile = blockIdx.x, slice = blockIdx.y, ntiles = gridDim.x;
  // zero both stages once: rows that are never written stay zero
  for (int i = tid; i < 2 * kStage / 16; i += kTcThreads) reinterpret_cast<uint4*>(stage0)[i] = make_uint4(0, 0, 0, 0);
  if (warp == 0) {
    tmem_alloc(tslot, 2 * kTcN);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = *tslot;
  // this thread's slice of the tile: TMEM lane quarter (warp % 4) and 64 of
  // the 256 columns (warp / 4); its running sum 256 columns further on
  const int q4 = warp & 3, h2 = warp >> 2;
  const uint32_t tcol = taddr + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(h2 * 64);
  {
    float z[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) z[i] = 0.f;
    tmem_st32(tcol + kTcN, z);
    tmem_st32(tcol + kTcN + 32, z);
  }
  const long long x0 = (long long)slice * kTcKC * chunks;
  const long long xend = (x0 + (long long)kTcKC * chunks < N3) ? x0 + (long long)kTcKC * chunks : N3;
  const int nch = x0 < xend ? (int)((xend - x0 + kTcKC - 1) / kTcKC) : 0;
  const uint32_t idesc = tc_idesc();
  // fixed roles
  const int rowA = tid & (kTcM - 1), kgA = tid / kTcM;
  const bool actA = rowA < nf;
  const int srcA = rowA * kTcRow + kgA * 8, dstA = canon_off(rowA, kgA);
  const int rowB = tid & (kTcN - 1), khB = tid / kTcN;
  short2 bc = make_short2(-1, -1);
  if (tile * kTcN + rowB < npairs) bc = pairs[tile * kTcN + rowB];
  const bool actB = bc.x >= 0;
  const int srcB1 = (actB ? bc.x : 0) * kTcRow + khB * 16, srcB2 = (actB ? bc.y : 0) * kTcRow + khB * 16;
  const int dstB0 = canon_off(rowB, 2 * khB), dstB1 = canon_off(rowB, 2 * khB + 1);
  const int cf0 = tid >> 3, cf1 = (tid + kTcThreads) >> 3, ck4 = (tid & 7) * 4;
  const bool cp0 = cf0 < nf, cp1 = cf1 < nf;
  const float* csrc0 = I + (size_t)(cp0 ? cf0 : 0) * N3;
  const float* csrc1 = I + (size_t)(cp1 ? cf1 : 0) * N3;
  const uint32_t cdst0 = smem_u32(Iring + cf0 * kTcRow + ck4), cdst1 = smem_u32(Iring + cf1 * kTcRow + ck4);
  bool ok = true;
  // asynchronous copies of a chunk's field values into its ring slot (16 bytes
  // each; points past the slice are zero-filled)
  auto prefetch = [&](int cc) {
    if (cc < nch) {
      const long long x = x0 + (long long)cc * kTcKC + ck4;
      const int bytes = x + 4 <= xend ? 16 : (x < xend ? (int)(xend - x) * 4 : 0);
      const long long xs = x < xend ? x : 0;
      const uint32_t so = (uint32_t)((cc % 3) * ring * 4);
      if (cp0)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(cdst0 + so), "l"(csrc0 + xs), "r"(bytes)
                     : "memory");
      if (cp1)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(cdst1 + so), "l"(csrc1 + xs), "r"(bytes)
                     : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  // drain of the run ending with chunk cl: wait for that chunk's MMAs, add
  // the tile to the running sum (ok is made block-uniform: tcgen05.ld is a
  // warp-collective)
  constexpr int kDrain = tc_drain<NS>();
  auto drain = [&](int cl) {
    const bool w = ok && mbar_wait(&bar[cl & 1], (uint32_t)((cl >> 1) & 1), err, 16);
    ok = __syncthreads_and(w) != 0;
    tc_fence_after();
    if (ok) {
      // per 32 columns: both loads, one wait, add, store; one store wait
#pragma unroll
      for (int cg = 0; cg < 2; ++cg) {
        uint32_t v[32], u[32];
        tmem_ld32_async(tcol + cg * 32, v);
        tmem_ld32_async(tcol + kTcN + cg * 32, u);
        tmem_wait_ld(v);
        tmem_wait_ld(u);
#pragma unroll
        for (int i = 0; i < 32; ++i) u[i] = __float_as_uint(__uint_as_float(u[i]) + __uint_as_float(v[i]));
        tmem_st32_async(tcol + kTcN + cg * 32, u);
      }
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
  };
  prefetch(0);
  prefetch(1);
  for (int c = 0; c < nch; ++c) {
    const int s = c & 1;
    unsigned char* st = stage0 + s * kStage;
    unsigned char* Ap = st;                      // NS tiles of kTcABytes
    unsigned char* Bp = st + NS * kTcABytes;     // NS tiles of kTcBBytes
    prefetch(c + 2);
    asm volatile("cp.async.wait_group 2;" ::: "memory");
    const float* Ist = Iring + (c % 3) * ring;
    // the MMAs that read this stage two chunks ago must have finished
    if (c >= 2 && ok) ok = mbar_wait(&bar[s], (uint32_t)(((c - 2) >> 1) & 1), err, 16);
    ok = __syncthreads_and(ok) != 0;
    // A: rows (l, a) = field index; a quarter-warp stores 8 consecutive rows
    // of one k-group (one contiguous, conflict-free 128-byte span)
    if (actA) {
      const float4 p = *reinterpret_cast<const float4*>(Ist + srcA);
      const float4 q = *reinterpret_cast<const float4*>(Ist + srcA + 4);
      const float v[8] = {p.x, p.y, p.z, p.w, q.x, q.y, q.z, q.w};
      uint4 parts[NS];
      split8<NS>(v, parts);
#pragma unroll
      for (int k = 0; k < NS; ++k) *reinterpret_cast<uint4*>(Ap + k * kTcABytes + dstA) = parts[k];
    }
    // B: rows = pairs (b, c) of this tile, products of the l = 0 fields
    if (actB) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float4 b0 = *reinterpret_cast<const float4*>(Ist + srcB1 + 8 * h);
        const float4 b1 = *reinterpret_cast<const float4*>(Ist + srcB1 + 8 * h + 4);
        const float4 c0 = *reinterpret_cast<const float4*>(Ist + srcB2 + 8 * h);
        const float4 c1 = *reinterpret_cast<const float4*>(Ist + srcB2 + 8 * h + 4);
        const float v[8] = {b0.x * c0.x, b0.y * c0.y, b0.z * c0.z, b0.w * c0.w,
                            b1.x * c1.x, b1.y * c1.y, b1.z * c1.z, b1.w * c1.w};
        uint4 parts[NS];
        split8<NS>(v, parts);
        const int d = h ? dstB1 : dstB0;
#pragma unroll
        for (int k = 0; k < NS; ++k) *reinterpret_cast<uint4*>(Bp + k * kTcBBytes + d) = parts[k];
      }
    }
    fence_proxy_async();
    __syncthreads();
    // a run ended with chunk c - 1: its MMAs ran while this chunk was built,
    // so the tensor pipe waits only for the drain, not for a build
    if (c > 0 && c % kDrain == 0) drain(c - 1);
    if (tid == 0 && ok) {
      tc_fence_after();
      // products (i, j) of A part i and B part j whose order is at most 2^-16
      constexpr int NP = NS == 2 ? 3 : 6;
      constexpr int pi[6] = {0, 0, 1, 0, 2, 1};
      constexpr int pj[6] = {0, 1, 0, 2, 0, 1};
#pragma unroll
      for (int ks = 0; ks < kTcKC / 16; ++ks) {
        // K step ks covers k-groups 2 ks and 2 ks + 1 (32 bytes further along the rows)
#pragma unroll
        for (int q = 0; q < NP; ++q) {
          const uint64_t ad = sdesc(Ap + pi[q] * kTcABytes + ks * 32, 16, 512);
          const uint64_t bd = sdesc(Bp + pj[q] * kTcBBytes + ks * 32, 16, 512);
          umma_bf16(taddr, ad, bd, idesc, ((c % kDrain) > 0 || ks > 0 || q > 0) ? 1u : 0u);
        }
      }
      umma_commit(&bar[s]);
    }
    // No barrier here: the next chunk builds the other stage, which the MMAs
    // of chunk c - 1 have released (mbarrier wait), and reads a ring slot the
    // copies of chunk c + 1 filled; stage s is rebuilt only after this commit.
  }
  if (nch > 0) drain(nch - 1);
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  // the last drain waited for every MMA of the slice
  float* dst = part + (((size_t)slice * ntiles + tile) * kTcM + q4 * 32 + (tid & 31)) * kTcN + h2 * 64;
#pragma unroll
  for (int cg = 0; cg < 2; ++cg) {
    float u[32];
    tmem_ld32(tcol + kTcN + cg * 32, u);
#pragma unroll
    for (int i = 0; i < 32; i += 4)
      *reinterpret_cast<float4*>(dst + cg * 32 + i) = make_float4(u[i], u[i + 1], u[i + 2], u[i + 3]);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(taddr, 2 * kTcN);
}

// out[t * 3 + li] = sum over slices of D[m = li * S + a][n = pair(b, c)].
__global__ void k_tc_reduce(const float* __restrict__ part, int nslices, int ntiles, const int* __restrict__ om,
                            const int* __restrict__ on, int nout, double* __restrict__ out) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= nout) return;
  const int m = om[o], n = on[o];
  if (m < 0) {
    out[o] = 0.0;
    return;
  }
  const int tile = n / kTcN, col = n - tile * kTcN;
  double s = 0.0;
  for (int k = 0; k < nslices; ++k) s += (double)part[(((size_t)k * ntiles + tile) * kTcM + m) * kTcN + col];
  out[o] = s;
}

template <int NS>
static size_t tc_smem_bytes(int nf) {
  return 2 * (size_t)tc_stage_bytes<NS>() + 3 * sizeof(float) * (size_t)nf * kTcRow + 2 * sizeof(uint64_t) + 16;
}

cudaError_t launch_contract_tc(const float* I, long long N3, int nf, int S, const short2* pairs, int npairs,
                               float* part, int* err, int nslices, int chunks, int nsplit, cudaStream_t s) {
  const int ntiles = (npairs + kTcN - 1) / kTcN;
  const dim3 grid(ntiles, nslices);
  if (nsplit == 2) {
    const size_t sm = tc_smem_bytes<2>(nf);
    raise_smem_limit((const void*)k_contract_tc<2>, sm);
    k_contract_tc<2><<<grid, kTcThreads, sm, s>>>(I, N3, nf, S, pairs, npairs, chunks, part, err);
  } else {
    const size_t sm = tc_smem_bytes<3>(nf);
    raise_smem_limit((const void*)k_contract_tc<3>, sm);
    k_contract_tc<3><<<grid, kTcThreads, sm, s>>>(I, N3, nf, S, pairs, npairs, chunks, part, err);
  }
  return cudaGetLastError();
}

cudaError_t launch_tc_reduce(const float* part, int nslices, int ntiles, const int* om, const int* on, int nout,
                             double* out, cudaStream_t s) {
  k_tc_reduce<<<(nout + 255) / 256, 256, 0, s>>>(part, nslices, ntiles, om, on, nout, out);
  return cudaGetLastError();
}

}  // namespace fkp
