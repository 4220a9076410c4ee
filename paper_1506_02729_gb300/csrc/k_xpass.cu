// k_xpass.cu - the x-pass of the power-spectrum path: moment fields built at the nodes about
// the observer (eqs. Qij, Qijkl, Qab), two real fields per complex pencil, FFT along x
// (shared helpers and layouts in k_fftpass.cuh).
#include "k_fftpass.cuh"

namespace fkp {

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
// PO (per-object line of sight): gq holds the NF moment fields, gridded from
// the catalogs with each object's x^, one after the other (N^3 each); the
// block packs rows of fields 2p and 2p + 1 into pencil p instead of forming
// the moments at the nodes.
template <int N_, int LMAX, bool PO = false>
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
    if constexpr (PO) return;
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
    if constexpr (PO) {
      const size_t N3 = (size_t)N * N * N, r0 = (size_t)row * N;
      for (int x = tid; x < N; x += NTX) {
#pragma unroll
        for (int p = 0; p < NP; ++p) {
          const float m0 = (float)(long long)__ldg(gq + (size_t)(2 * p) * N3 + r0 + x) * kFixInvF;
          const float m1 = 2 * p + 1 < NF ? (float)(long long)__ldg(gq + (size_t)(2 * p + 1) * N3 + r0 + x) * kFixInvF
                                          : 0.f;
          A[ilv<NP, SWZ>(x, p)] = make_float2(m0, m1);
        }
      }
    }
    for (int x = tid; x < N && !PO; x += NTX) {
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

template <int N_, int LMAX, bool PO = false>
static cudaError_t xrun(const unsigned long long* gq, const float* gf, const GeomDev& g, const FftPlan& fp,
                        const float2* tw, float2* S1, int nsm, cudaStream_t s, int xm, const MockBatch& mb) {
  constexpr int NP = (nfields_of(LMAX) + 1) / 2;
  const size_t sm = xsm(g.N, NP);
  raise_smem_limit((const void*)k_xpass2<N_, LMAX, PO>, sm);
  int occ = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_xpass2<N_, LMAX, PO>, 32 * NP, sm);
  int grid = nsm * (occ > 0 ? occ : 1) * (xm > 0 ? xm : 2);
  if (grid > g.N * g.N) grid = g.N * g.N;
  k_xpass2<N_, LMAX, PO><<<dim3(grid, 1, mb.n), dim3(NP, 32), sm, s>>>(gq, gf, g, fp, tw, S1, mb);
  return cudaGetLastError();
}

template <int LMAX>
static cudaError_t xdispatch(const unsigned long long* gq, const float* gf, const GeomDev& g, const FftPlan& fp,
                             const float2* tw, float2* S1, int nsm, cudaStream_t s, int xm, const MockBatch& mb,
                             bool po) {
  // the per-object variant: the runtime-size kernel, whatever N
  if (po) return xrun<0, LMAX, true>(gq, gf, g, fp, tw, S1, nsm, s, xm, mb);
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
                         MockBatch mb, bool per_object) {
  if (per_object && (!gq || gf || mb.n != 1)) return cudaErrorInvalidValue;
  if (mt.nfields == nfields_of(4)) return xdispatch<4>(gq, gf, g, fp, tw, S1, nsm, s, xm, mb, per_object);
  if (mt.nfields == nfields_of(2)) return xdispatch<2>(gq, gf, g, fp, tw, S1, nsm, s, xm, mb, per_object);
  return xdispatch<0>(gq, gf, g, fp, tw, S1, nsm, s, xm, mb, per_object);
}

}  // namespace fkp
