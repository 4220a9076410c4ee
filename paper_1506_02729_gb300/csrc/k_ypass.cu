// k_ypass.cu - the y-pass of the power-spectrum path: FFT along y and the k_x, k_y
// polynomials of eqs. delta2b and delta4b summed into the k_z-power groups
// (shared helpers and layouts in k_fftpass.cuh).
#include "k_fftpass.cuh"

namespace fkp {

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
  // the polynomial coefficients a[o][j] of every member (in read order) for
  // this block's 8 columns, [member][o][j][c]: computed once per block instead
  // of once per member and thread
  float* coef = reinterpret_cast<float*>(tw + N);
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
  int total = 0;
  for (int s = 0; s < mt.nsweeps; ++s) total += mt.s_nmem[s];
  for (int e = tid; e < total * 10 * kT; e += NT) {
    const int cc = e % kT, oj = (e / kT) % 10, mi = e / (10 * kT), o = oj / 5, j = oj - 5 * o;
    int sw = 0, m = mi;
    while (m >= mt.s_nmem[sw]) m -= mt.s_nmem[sw++];
    const float nxc = (float)(blockIdx.x * kT + cc);
    float v = 0.f;
#pragma unroll
    for (int t = 0; t < 2; ++t)
      if (mt.s_j[sw][m][o][t] == j) v += mt.s_c[sw][m][o][t] * powi(nxc, mt.s_i[sw][m][o][t]);
    coef[e] = v;
  }
  __syncthreads();
  auto src_of = [&](int q) { return S1 + (size_t)q * fsz + ((size_t)z * NXT + xt) * tile; };
  if (tid == 0) {
    mbar_expect_tx(&bar[0], bytes);
    tma_load_1d(buf0, src_of(mt.s_field[0][0]), bytes, &bar[0]);
  }
  const int c = threadIdx.x, run = threadIdx.y;
  const int rl = (N + PassShape<NT>::kRun - 1) / PassShape<NT>::kRun;
  const int kx = xt * kT + c;
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
      // coefficients a[o][j] of n_y^j for this member and column
      float a[2][5];
#pragma unroll
      for (int o = 0; o < 2; ++o)
#pragma unroll
        for (int j = 0; j < 5; ++j) a[o][j] = coef[(it * 10 + o * 5 + j) * kT + c];
      // the member's value at k_y = i kRun + run, times its polynomials in n_y,
      // joins the thread's sums
      auto accumulate = [&](int i, float2 v) {
        const int ky = i * PassShape<NT>::kRun + run;
        const float ny = (float)smode(ky, N);
        const float s0 = fmaf(fmaf(fmaf(fmaf(a[0][4], ny, a[0][3]), ny, a[0][2]), ny, a[0][1]), ny, a[0][0]);
        acc0[i].x = fmaf(s0, v.x, acc0[i].x);
        acc0[i].y = fmaf(s0, v.y, acc0[i].y);
        if (nout > 1) {
          const float s1 = fmaf(fmaf(fmaf(fmaf(a[1][4], ny, a[1][3]), ny, a[1][2]), ny, a[1][1]), ny, a[1][0]);
          acc1[i].x = fmaf(s1, v.x, acc1[i].x);
          acc1[i].y = fmaf(s1, v.y, acc1[i].y);
        }
      };
      mbar_wait(&bar[cur], (uint32_t)((it >> 1) & 1), err, 4);
      if constexpr (fft_fusable<N_, kT, NT>()) {
        // the last FFT stage's butterflies produce exactly this thread's k_y
        // (y + i kRun): they are summed from registers, never stored
        fft_ct_fused<N_, kT, NT, -1, false, false>(bc, work, tw, accumulate);
      } else {
        const float2* R = fft_any<N_, kT, NT, -1>(bc, work, fp, tw);
#pragma unroll
        for (int i = 0; i < PassShape<NT>::kRL; ++i) {
          const int ky = i * PassShape<NT>::kRun + run;
          if (i < rl && ky < N) accumulate(i, R[ky * kT + c]);
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
// launch wrapper
// ----------------------------------------------------------------------------

template <int N_, int NT>
static cudaError_t yrun_nt(const float2* S1, const unsigned long long* gq, const float* gf, const GeomDev& g,
                           const MomentTable& mt, const FftPlan& fp, const float2* tw, float2* S2, int* err,
                           cudaStream_t s, const MockBatch& mb) {
  int total = 0;
  for (int q = 0; q < mt.nsweeps; ++q) total += mt.s_nmem[q];
  const size_t sm = ysm(g.N) + sizeof(float) * 10 * kT * (size_t)total;
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

}  // namespace fkp
