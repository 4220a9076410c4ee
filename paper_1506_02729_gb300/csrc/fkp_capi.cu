// fkp_capi.cu - the C ABI of include/fkp.h: contexts, plans (validation,
// FP64 look-up tables, twiddles, workspace) and the host-side sequencing of
// the kernels on one CUDA stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <initializer_list>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/fkp.h"
#include <map>
#include <mutex>
#include <utility>

#include "fkp_internal.h"

using namespace fkp;

// ----------------------------------------------------------------------------
// errors
// ----------------------------------------------------------------------------

static thread_local std::string g_last_error;

int fkp::set_error(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

cudaError_t fkp::raise_smem_limit(const void* func, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> limit;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  size_t& cur = limit[{func, dev}];
  if (bytes <= cur) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

extern "C" const char* fkp_last_error(void) { return g_last_error.c_str(); }
extern "C" const char* fkp_version(void) { return "fkp-gb300 0.1 (sm_103a)"; }

#define CK(call)                                                                                \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess)                                                                      \
      return set_error(FKP_ECUDA, "%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
  } while (0)

// ----------------------------------------------------------------------------
// context
// ----------------------------------------------------------------------------

extern "C" int fkp_context_create(int device, size_t hbm_budget_bytes, void** out) {
  if (!out) return set_error(FKP_EINVAL, "fkp_context_create: out is NULL");
  int ndev = 0;
  CK(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return set_error(FKP_EINVAL, "fkp_context_create: bad device %d", device);
  CK(cudaSetDevice(device));
  auto* c = new Context();
  c->device = device;
  c->budget = hbm_budget_bytes;
  CK(cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, device));
  *out = c;
  return FKP_OK;
}

extern "C" void fkp_context_destroy(void* ctx) { delete static_cast<Context*>(ctx); }

// ----------------------------------------------------------------------------
// plan
// ----------------------------------------------------------------------------

static bool radix_plan(int n, FftPlan& p) {
  p.n = n;
  p.nst = 0;
  int m = n;
  auto push = [&](int r) {
    if (p.nst >= 8) return false;
    p.radix[p.nst++] = r;
    return true;
  };
  while (m % 8 == 0) { if (!push(8)) return false; m /= 8; }
  while (m % 4 == 0) { if (!push(4)) return false; m /= 4; }
  while (m % 2 == 0) { if (!push(2)) return false; m /= 2; }
  while (m % 5 == 0) { if (!push(5)) return false; m /= 5; }
  while (m % 3 == 0) { if (!push(3)) return false; m /= 3; }
  return m == 1;
}

// Field list, y-pass sweeps and k_z-power groups for multipoles up to lmax
// (0, 2 or 4).
//
// Fields: grid * xh_x^i xh_y^j xh_z^k for F_0, the rank-2 components with at
// most one z (xx xy yy xz yz), the rank-4 ones with at most one z (xxxx xxxy
// xxyy xyyy yyyy xxxz xxyz xyyz yyyz) and zzzz: 16 instead of 1 + 6 + 15.  The
// others follow from the trace identities of the unit vector xh (eqs. Qij,
// Qijkl): sum_a Q_aa = F_0 and sum_c Q_abcc = Q_ab, so
//   Q_zz = F_0 - Q_xx - Q_yy,   Q_abzz = Q_ab - Q_abxx - Q_abyy.
// With S_2 = sum_ab k_a k_b Q_ab and S_4 = sum_abcd k_a k_b k_c k_d Q_abcd
// (the multiplicities 1, 2 of eq. delta2b and 1, 4, 6, 12 of eq. delta4b):
//   S_2 = A + nz G21 + nz^2 (F_0 - T)
//   S_4 = G40 + nz G41 + nz^2 (6 A - U) + nz^3 (2 G21 - W) + nz^4 Q_zzzz
// where
//   A   = nx^2 Qxx + 2 nx ny Qxy + ny^2 Qyy            T = Qxx + Qyy
//   G21 = 2 nx Qxz + 2 ny Qyz
//   G40 = nx^4 Qxxxx + 4 nx^3 ny Qxxxy + 6 nx^2 ny^2 Qxxyy + 4 nx ny^3 Qxyyy + ny^4 Qyyyy
//   U   = 6 nx^2 (Qxxxx + Qxxyy) + 12 nx ny (Qxxxy + Qxyyy) + 6 ny^2 (Qxxyy + Qyyyy)
//   G41 = 4 nx^3 Qxxxz + 12 nx^2 ny Qxxyz + 12 nx ny^2 Qxyyz + 4 ny^3 Qyyyz
//   W   = 4 nx (Qxxxz + Qxyyz) + 4 ny (Qxxyz + Qyyyz).
// The y-pass forms the nine groups (F_0, A, T, G21, G40, U, G41, W, Q_zzzz)
// after its FFT; the z-pass applies the powers of nz after its own.  At the
// observer's own node xh = 0, where Qxx + Qyy + Qzz = 0 rather than F_0: the
// y-pass adds that node's F to T, which keeps F_0 - T equal to Q_zz there too.
void fkp::build_moments(int lmax, MomentTable& mt) {
  memset(&mt, 0, sizeof(mt));
  enum { F0 = 0, XX, XY, YY, XZ, YZ, XXXX, XXXY, XXYY, XYYY, YYYY, XXXZ, XXYZ, XYYZ, YYYZ, ZZZZ };
  static const unsigned char ex[16][3] = {{0, 0, 0}, {2, 0, 0}, {1, 1, 0}, {0, 2, 0}, {1, 0, 1}, {0, 1, 1},
                                          {4, 0, 0}, {3, 1, 0}, {2, 2, 0}, {1, 3, 0}, {0, 4, 0}, {3, 0, 1},
                                          {2, 1, 1}, {1, 2, 1}, {0, 3, 1}, {0, 0, 4}};
  mt.nfields = lmax >= 4 ? 16 : (lmax >= 2 ? 6 : 1);
  for (int q = 0; q < mt.nfields; ++q)
    for (int a = 0; a < 3; ++a) mt.e[q][a] = ex[q][a];
  int ns = 0, ng = 0;
  // one sweep: its fields, then (output, member, term) = c nx^i ny^j
  auto sweep = [&](std::initializer_list<int> fields, int nout, int obs) {
    for (int f : fields) mt.s_field[ns][mt.s_nmem[ns]++] = f;
    mt.s_nout[ns] = nout;
    mt.s_obs[ns] = obs;
    for (int o = 0; o < nout; ++o) mt.s_out[ns][o] = ng++;
    return ns++;
  };
  auto term = [&](int s, int m, int o, int t, float cf, int i, int j) {
    mt.s_c[s][m][o][t] = cf;
    mt.s_i[s][m][o][t] = (unsigned char)i;
    mt.s_j[s][m][o][t] = (unsigned char)j;
  };
  auto group = [&](int g, int f0, float c2, int p2, float c4, int p4) {
    mt.g_f0[g] = f0;
    mt.g_c2[g] = c2;
    mt.g_p2[g] = (unsigned char)p2;
    mt.g_c4[g] = lmax >= 4 ? c4 : 0.f;
    mt.g_p4[g] = (unsigned char)p4;
  };
  int s = sweep({F0}, 1, -1);
  term(s, 0, 0, 0, 1.f, 0, 0);
  group(0, 1, lmax >= 2 ? 1.f : 0.f, 2, 0.f, 0);
  if (lmax >= 2) {
    s = sweep({XX, XY, YY}, 2, 1);                                   // A, T
    term(s, 0, 0, 0, 1.f, 2, 0); term(s, 1, 0, 0, 2.f, 1, 1); term(s, 2, 0, 0, 1.f, 0, 2);
    term(s, 0, 1, 0, 1.f, 0, 0); term(s, 2, 1, 0, 1.f, 0, 0);
    group(1, 0, 1.f, 0, 6.f, 2);
    group(2, 0, -1.f, 2, 0.f, 0);
    s = sweep({XZ, YZ}, 1, -1);                                      // G21
    term(s, 0, 0, 0, 2.f, 1, 0); term(s, 1, 0, 0, 2.f, 0, 1);
    group(3, 0, 1.f, 1, 2.f, 3);
  }
  if (lmax >= 4) {
    s = sweep({XXXX, XXXY, XXYY, XYYY, YYYY}, 2, -1);                // G40, U
    term(s, 0, 0, 0, 1.f, 4, 0); term(s, 1, 0, 0, 4.f, 3, 1); term(s, 2, 0, 0, 6.f, 2, 2);
    term(s, 3, 0, 0, 4.f, 1, 3); term(s, 4, 0, 0, 1.f, 0, 4);
    term(s, 0, 1, 0, 6.f, 2, 0); term(s, 1, 1, 0, 12.f, 1, 1); term(s, 2, 1, 0, 6.f, 2, 0);
    term(s, 2, 1, 1, 6.f, 0, 2); term(s, 3, 1, 0, 12.f, 1, 1); term(s, 4, 1, 0, 6.f, 0, 2);
    group(4, 0, 0.f, 0, 1.f, 0);
    group(5, 0, 0.f, 0, -1.f, 2);
    s = sweep({XXXZ, XXYZ, XYYZ, YYYZ}, 2, -1);                      // G41, W
    term(s, 0, 0, 0, 4.f, 3, 0); term(s, 1, 0, 0, 12.f, 2, 1); term(s, 2, 0, 0, 12.f, 1, 2);
    term(s, 3, 0, 0, 4.f, 0, 3);
    term(s, 0, 1, 0, 4.f, 1, 0); term(s, 1, 1, 0, 4.f, 0, 1); term(s, 2, 1, 0, 4.f, 1, 0);
    term(s, 3, 1, 0, 4.f, 0, 1);
    group(6, 0, 0.f, 0, 1.f, 1);
    group(7, 0, 0.f, 0, -1.f, 3);
    s = sweep({ZZZZ}, 1, -1);                                        // Q_zzzz
    term(s, 0, 0, 0, 1.f, 0, 0);
    group(8, 0, 0.f, 0, 1.f, 4);
  }
  mt.nsweeps = ns;
  mt.ngroups = ng;
}

// The table reproduces S_2 = (k.xh)^2 and S_4 = (k.xh)^4 (F = 1) for unit
// vectors xh and arbitrary k: a check of every coefficient above.
bool fkp::moments_identities_hold(const MomentTable& mt, int lmax) {
  unsigned long long st = 0x9E3779B97F4A7C15ull;
  auto rnd = [&]() {
    st = st * 6364136223846793005ull + 1442695040888963407ull;
    return (double)(st >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
  };
  for (int trial = 0; trial < 16; ++trial) {
    double h[3] = {rnd(), rnd(), rnd()}, k[3] = {8 * rnd(), 8 * rnd(), 8 * rnd()};
    const double hn = std::sqrt(h[0] * h[0] + h[1] * h[1] + h[2] * h[2]);
    for (double& v : h) v /= hn;
    double f[kMaxFields], out[kMaxGroups] = {0};
    for (int q = 0; q < mt.nfields; ++q)
      f[q] = std::pow(h[0], mt.e[q][0]) * std::pow(h[1], mt.e[q][1]) * std::pow(h[2], mt.e[q][2]);
    for (int s = 0; s < mt.nsweeps; ++s)
      for (int m = 0; m < mt.s_nmem[s]; ++m)
        for (int o = 0; o < mt.s_nout[s]; ++o)
          for (int t = 0; t < 2; ++t)
            out[mt.s_out[s][o]] += mt.s_c[s][m][o][t] * std::pow(k[0], mt.s_i[s][m][o][t]) *
                                   std::pow(k[1], mt.s_j[s][m][o][t]) * f[mt.s_field[s][m]];
    double F0 = 0, S2 = 0, S4 = 0;
    for (int g = 0; g < mt.ngroups; ++g) {
      if (mt.g_f0[g]) F0 += out[g];
      S2 += mt.g_c2[g] * std::pow(k[2], mt.g_p2[g]) * out[g];
      S4 += mt.g_c4[g] * std::pow(k[2], mt.g_p4[g]) * out[g];
    }
    const double kh = k[0] * h[0] + k[1] * h[1] + k[2] * h[2];
    const double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
    if (std::fabs(F0 - 1.0) > 1e-12) return false;
    if (lmax >= 2 && std::fabs(S2 - kh * kh) > 1e-9 * k2) return false;
    if (lmax >= 4 && std::fabs(S4 - kh * kh * kh * kh) > 1e-9 * k2 * k2) return false;
  }
  return true;
}

extern "C" int fkp_check_tables(void) {
  for (int lmax = 0; lmax <= 4; lmax += 2) {
    MomentTable mt;
    build_moments(lmax, mt);
    if (!moments_match(mt)) return set_error(FKP_ESTATE, "moment table for lmax=%d does not match the kernels", lmax);
    if (!moments_identities_hold(mt, lmax))
      return set_error(FKP_ESTATE, "moment table for lmax=%d does not reproduce S_2, S_4", lmax);
  }
  return FKP_OK;
}

// The grid node where the kernels' FP32 node position relative to the
// observer, fmaf(i, H, origin - observer) per axis, is exactly zero (x^ = 0
// there), or -1 on every axis when there is none.
void fkp::observer_node(GeomDev& g) {
  g.obs_x = g.obs_y = g.obs_z = -1;
  if (g.los_inf) return;
  auto axis = [&](float r) {
    for (int i = 0; i < g.N; ++i)
      if (std::fmaf((float)i, g.H, r) == 0.f) return i;
    return -1;
  };
  const int ix = axis(g.rx), iy = axis(g.ry), iz = axis(g.rz);
  if (ix >= 0 && iy >= 0 && iz >= 0) {
    g.obs_x = ix;
    g.obs_y = iy;
    g.obs_z = iz;
  }
}

static bool smooth235(int n) {
  if (n <= 0) return false;
  for (int f : {2, 3, 5}) while (n % f == 0) n /= f;
  return n == 1;
}

void* fkp::Plan::alloc(size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
  buffers.push_back(p);
  bytes_total += bytes;
  return p;
}

fkp::Plan::~Plan() {
  if (graph_exec) cudaGraphExecDestroy(graph_exec);
  if (cap_stream) cudaStreamDestroy(cap_stream);
  bisp_plan_free(this);
  for (void* p : buffers) cudaFree(p);
  for (void* p : staging) cudaFree(p);
  if (d_xyzv) cudaFree(d_xyzv);
  if (d_vw2) cudaFree(d_vw2);
  if (h_pinned) cudaFreeHost(h_pinned);
  if (batch_mem) cudaFree(batch_mem);
  for (auto& e : ev) if (e) cudaEventDestroy(e);
  if (ev_fork) cudaEventDestroy(ev_fork);
  if (ev_join) cudaEventDestroy(ev_join);
  if (side) cudaStreamDestroy(side);
}

// z-pass threads per block for a grid: 256 (two blocks per SM) up to 256^3,
// 512 (one per SM: its three accumulators per point need the registers) above.
int fkp::z_threads_for(int N) { return N <= 256 ? 256 : 512; }

// Times the candidate launch schedules of the three FFT passes on the plan's
// own workspace (zeroed: the passes' cost does not depend on the values) and
// keeps the fastest of each; the choice is shared by later plans of the same
// grid and multipole order in this context.  About 12 launches of each pass,
// once per (N, lmax).
static int tune_schedule(Plan* P) {
  const std::pair<int, int> key{P->g.N, P->lmax};
  std::lock_guard<std::mutex> lk(P->ctx->tune_mu);
  auto it = P->ctx->schedules.find(key);
  if (it != P->ctx->schedules.end()) {
    P->sched = it->second;
    return FKP_OK;
  }
  const int N = P->g.N;
  const size_t N3 = (size_t)N * N * N, half = field_elems(N) * sizeof(float2);
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  int rc = FKP_OK;
  auto fail = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess && rc == FKP_OK) rc = set_error(FKP_ECUDA, "schedule tuning (%s): %s", what, cudaGetErrorString(e));
    return e != cudaSuccess;
  };
  if (!fail(cudaEventCreate(&e0), "event") && !fail(cudaEventCreate(&e1), "event")) {
    fail(cudaMemsetAsync(P->d_grid, 0, N3 * 8, s), "memset");
    fail(cudaMemsetAsync(P->d_S1, 0, half * P->mt.nfields, s), "memset");
    fail(cudaMemsetAsync(P->d_S2, 0, half * P->mt.ngroups, s), "memset");
    fail(cudaMemsetAsync(P->d_err, 0, sizeof(int) * 4, s), "memset");
    ZParams zp{};
    zp.nbins = P->pb.nbins;
    zp.lmax = P->lmax;
    zp.kf = (float)(2.0 * M_PI / P->geom.L);
    zp.lut = P->d_lut;
    zp.winv = P->d_winv;
    zp.mode = 0;
    // mean time of 3 launches after one warm-up launch
    auto timed = [&](auto&& launch, const char* what) -> float {
      if (rc || fail(launch(), what)) return 1e30f;
      fail(cudaEventRecord(e0, s), "event");
      for (int r = 0; r < 3; ++r) fail(launch(), what);
      fail(cudaEventRecord(e1, s), "event");
      float ms = 1e30f;
      if (!fail(cudaEventSynchronize(e1), what)) fail(cudaEventElapsedTime(&ms, e0, e1), "event");
      return ms / 3.f;
    };
    PassSchedule best;
    float bx = 1e30f, by = 1e30f, bz = 1e30f;
    for (int xm : {1, 2, 4, 8}) {
      const float t = timed([&] { return launch_xpass(P->d_grid, nullptr, P->g, P->mt, P->fp, P->d_tw, P->d_S1,
                                                      P->ctx->nsm, s, xm); }, "x-pass");
      if (t < bx) { bx = t; best.x_mult = xm; }
    }
    for (int nt : {256, 512}) {
      const float t = timed([&] { return launch_ypass(P->d_S1, P->d_grid, nullptr, P->g, P->mt, P->fp, P->d_tw,
                                                      P->d_S2, P->d_err + 1, s, nt); }, "y-pass");
      if (t < by) { by = t; best.y_threads = nt; }
    }
    // the z-pass block shape sets the partition of each k_z column into the
    // FP32 runs of the bin sums, so it is fixed per grid rather than tuned:
    // results then do not depend on the tuning (bit for bit)
    best.z_threads = z_threads_for(N);
    bz = timed([&] { return launch_zpass(P->d_S2, P->g, P->mt, P->fp, P->d_tw, zp, P->d_zpart, P->d_zpartc,
                                         P->d_err + 1, s, P->ctx->nsm, best.z_threads); }, "z-pass");
    best.ms[0] = bx;
    best.ms[1] = by;
    best.ms[2] = bz;
    best.tuned = true;
    if (rc == FKP_OK) {
      P->sched = best;
      P->ctx->schedules[key] = best;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  cudaStreamDestroy(s);
  return rc;
}

extern "C" int fkp_plan_schedule(const void* plan, int* x_mult, int* y_threads, int* z_threads, float* tuned_ms) {
  const auto* P = static_cast<const Plan*>(plan);
  if (!P) return set_error(FKP_EINVAL, "NULL plan");
  if (x_mult) *x_mult = P->sched.x_mult;
  if (y_threads) *y_threads = P->sched.y_threads;
  if (z_threads) *z_threads = P->sched.z_threads;
  if (tuned_ms)
    for (int i = 0; i < 3; ++i) tuned_ms[i] = P->sched.tuned ? P->sched.ms[i] : 0.f;
  return FKP_OK;
}

extern "C" int fkp_plan_set_schedule(void* plan, int x_mult, int y_threads, int z_threads) {
  auto* P = static_cast<Plan*>(plan);
  if (!P) return set_error(FKP_EINVAL, "NULL plan");
  if ((x_mult != 1 && x_mult != 2 && x_mult != 4 && x_mult != 8) || (y_threads != 256 && y_threads != 512) ||
      (z_threads != 256 && z_threads != 512))
    return set_error(FKP_EINVAL, "schedule: x_mult in {1, 2, 4, 8}, y_threads and z_threads in {256, 512}");
  P->sched.x_mult = x_mult;
  P->sched.y_threads = y_threads;
  P->sched.z_threads = z_threads;
  if (P->graph_exec) cudaGraphExecDestroy(P->graph_exec);  // captured with the old launches
  P->graph_exec = nullptr;
  P->last_valid = false;
  bisp_drop_graph(P);
  return FKP_OK;
}

extern "C" int fkp_plan_create(void* vctx, const fkp_geometry_t* geom, const fkp_pbins_t* pb,
                               const fkp_bshells_t* bs, uint32_t want, void** out) {
  auto* ctx = static_cast<Context*>(vctx);
  if (!ctx || !geom || !pb || !out) return set_error(FKP_EINVAL, "fkp_plan_create: NULL argument");
  const int N = geom->N;
  if (N < 8 || N > 512 || (N & 1) || !smooth235(N))
    return set_error(FKP_EINVAL, "grid N=%d must be even, 8 <= N <= 512 and a product of 2, 3, 5", N);
  if (geom->assign < 2 || geom->assign > 4)
    return set_error(FKP_EINVAL, "assign must be 2 (CIC), 3 (TSC) or 4 (PCS)");
  if (!(geom->L > 0)) return set_error(FKP_EINVAL, "box side L must be positive");
  if (pb->nbins < 1 || pb->nbins > kMaxBins || !(pb->dk > 0) || !(pb->kmin >= 0))
    return set_error(FKP_EINVAL, "bad P bins (nbins in [1,%d], dk > 0, kmin >= 0)", kMaxBins);
  const bool wantB = (want & (FKP_B0 | FKP_B2 | FKP_B4 | FKP_B4B)) != 0;
  if (wantB) {
    if (!bs || bs->nshells < 1 || bs->nshells > kMaxShells || bs->width < 1 || bs->step < 1 ||
        bs->first < 1 || 2 * bs->first < bs->width)
      return set_error(FKP_EINVAL, "bad bispectrum shells");
    const double nmax = bs->first + (bs->nshells - 1) * (double)bs->step + 0.5 * bs->width;
    if (3.0 * nmax >= N) return set_error(FKP_EGEOM, "3*n_max = %.1f >= N = %d: triangle sums would alias", 3 * nmax, N);
    if (nmax >= N / 2) return set_error(FKP_EGEOM, "shells reach the Nyquist plane");
  }
  if ((want & FKP_XHAT_OBJECT) && (wantB || geom->interlace))
    return set_error(FKP_EINVAL, "FKP_XHAT_OBJECT: power multipoles of one grid only (no FKP_B*, no interlace)");
  if (geom->observer_at_infinity) {
    const double l2 = geom->los[0] * geom->los[0] + geom->los[1] * geom->los[1] + geom->los[2] * geom->los[2];
    if (!(l2 > 0)) return set_error(FKP_EINVAL, "los must be nonzero when the observer is at infinity");
  }
  CK(cudaSetDevice(ctx->device));
  auto* P = new Plan();
  P->ctx = ctx;
  P->geom = *geom;
  P->pb = *pb;
  if (bs) P->bs = *bs;
  P->want = want;
  P->wantB = wantB;
  P->per_object = (want & FKP_XHAT_OBJECT) != 0;
  int lmax = 0;
  if (want & (FKP_P2 | FKP_P4B | FKP_B2 | FKP_B4B)) lmax = 2;
  if (want & (FKP_P4 | FKP_B4 | FKP_P6B | FKP_P8B)) lmax = 4;
  P->lmax = lmax;
  build_moments(lmax, P->mt);
  if (!moments_match(P->mt) || !moments_identities_hold(P->mt, lmax)) {
    delete P;
    return set_error(FKP_ESTATE, "internal: moment table inconsistent");
  }
  if (!radix_plan(N, P->fp)) { delete P; return set_error(FKP_EINVAL, "no radix plan for N=%d", N); }

  // geometry as the kernels see it
  GeomDev& g = P->g;
  g.N = N;
  g.NH = N / 2 + 1;
  g.H = (float)(geom->L / N);
  g.invH = (float)(N / geom->L);
  g.ox = (float)geom->origin[0];
  g.oy = (float)geom->origin[1];
  g.oz = (float)geom->origin[2];
  g.rx = (float)(geom->origin[0] - geom->observer[0]);
  g.ry = (float)(geom->origin[1] - geom->observer[1]);
  g.rz = (float)(geom->origin[2] - geom->observer[2]);
  g.los_inf = geom->observer_at_infinity ? 1 : 0;
  {
    const double l = std::sqrt(geom->los[0] * geom->los[0] + geom->los[1] * geom->los[1] + geom->los[2] * geom->los[2]);
    g.lx = l > 0 ? (float)(geom->los[0] / l) : 0.f;
    g.ly = l > 0 ? (float)(geom->los[1] / l) : 0.f;
    g.lz = l > 0 ? (float)(geom->los[2] / l) : 1.f;
  }
  g.assign = geom->assign;
  g.periodic = geom->periodic ? 1 : 0;
  g.P_fkp = (float)geom->P_fkp;
  g.P_fkp_lo = (float)(geom->P_fkp - (double)g.P_fkp);
  g.alpha_mode = geom->alpha_mode;
  observer_node(g);
  // with each object's x^ the moment fields obey the trace identity object by
  // object, so the node at the observer needs no correction
  if (P->per_object) g.obs_x = g.obs_y = g.obs_z = -1;
  P->interlace = geom->interlace != 0;
  if (P->interlace) {
    // the second grid: nodes at origin + (i + 1/2) H
    GeomDev& h = P->g2;
    h = g;
    const double half = 0.5 * geom->L / N;
    h.ox = (float)(geom->origin[0] + half);
    h.oy = (float)(geom->origin[1] + half);
    h.oz = (float)(geom->origin[2] + half);
    h.rx = (float)(geom->origin[0] + half - geom->observer[0]);
    h.ry = (float)(geom->origin[1] + half - geom->observer[1]);
    h.rz = (float)(geom->origin[2] + half - geom->observer[2]);
    observer_node(h);
  }

  // FP64 tables on the host
  const double kf = 2.0 * M_PI / geom->L;
  const int n2max = 3 * (N / 2) * (N / 2);
  std::vector<short> lut(n2max + 1, -1);
  double min_gap = 1e300;
  for (int n2 = 1; n2 <= n2max; ++n2) {
    const double k = kf * std::sqrt((double)n2);
    long b = (long)std::floor((k - pb->kmin) / pb->dk);
    if (b < -1) b = -1;
    if (b > pb->nbins) b = pb->nbins;
    while (b >= 0 && k < pb->kmin + pb->dk * b) --b;
    while (b < pb->nbins && b >= -1 && k >= pb->kmin + pb->dk * (b + 1)) ++b;
    if (b >= 0 && b < pb->nbins) {
      lut[n2] = (short)b;
      const double lo = pb->kmin + pb->dk * b, hi = pb->kmin + pb->dk * (b + 1);
      min_gap = std::min(min_gap, std::min(std::fabs(k - lo), std::fabs(hi - k)) / k);
    }
  }
  P->min_edge_gap = min_gap;
  std::vector<float2> tw(N);
  for (int m = 0; m < N; ++m) {
    const double a = 2.0 * M_PI * (double)m / (double)N;
    tw[m] = make_float2((float)std::cos(a), (float)-std::sin(a));
  }
  std::vector<float> winv(3 * N, 1.0f);
  if (geom->compensate) {
    for (int i = 0; i < N; ++i) {
      const int n = i <= N / 2 ? i : i - N;
      const double t = M_PI * n / N;
      const double s = n == 0 ? 1.0 : std::sin(t) / t;
      const double w = std::pow(s, geom->assign);
      for (int a = 0; a < 3; ++a) winv[a * N + i] = (float)(1.0 / w);
    }
  }
  std::vector<float2> hph(N);  // e^{-i pi n/N}, n the signed index of i
  for (int i = 0; i < N; ++i) {
    const int n = i <= N / 2 ? i : i - N;
    const double a = M_PI * (double)n / (double)N;
    hph[i] = make_float2((float)std::cos(a), (float)-std::sin(a));
  }

  // device workspace
  const size_t N3 = (size_t)N * N * N;
  const size_t half = field_elems(N);  // one tile-major half spectrum, k_x padded to tiles of 8
  P->nblk_cat = std::max(1, ctx->nsm * 8);
  P->nblk_z = yz_tiles(N) * N;
  bool ok = true;
  auto A = [&](size_t bytes) { void* p = P->alloc(bytes); if (!p) ok = false; return p; };
  P->d_grid = (unsigned long long*)A(N3 * 8 * (P->per_object ? (size_t)P->mt.nfields : 1));
  if (wantB) P->d_gridw = (unsigned long long*)A(N3 * 8);
  if (P->interlace) {
    P->d_grid2 = (unsigned long long*)A(N3 * 8);
    if (wantB) P->d_gridw2 = (unsigned long long*)A(N3 * 8);
  }
  P->d_hph = (float2*)A(sizeof(float2) * N);
  P->d_S1 = (float2*)A(half * sizeof(float2) * P->mt.nfields);
  P->d_S2 = (float2*)A(half * sizeof(float2) * P->mt.ngroups * (P->interlace ? 2 : 1));
  P->d_tw = (float2*)A(sizeof(float2) * N);
  P->d_lut = (short*)A(sizeof(short) * (n2max + 1));
  P->d_winv = (float*)A(sizeof(float) * 3 * N);
  P->d_scpart = (double*)A(sizeof(double) * SC_NSUM * 2 * P->nblk_cat);
  P->d_labpart = (double*)A(sizeof(double) * LAB_NSUM * P->nblk_cat);
  P->d_ds = (double*)A(sizeof(double) * (DS_COUNT + LAB_NSUM + 8));
  P->d_err = (int*)A(sizeof(int) * 4);
  {
    const int ntx = assign_tiles_per_axis(N);
    P->ntiles = ntx * ntx * ntx;
  }
  P->d_tcnt = (int*)A(sizeof(int) * P->ntiles);
  P->d_toff = (int*)A(sizeof(int) * (P->ntiles + 1));
  P->d_titem = (int*)A(sizeof(int) * (P->ntiles + 1));
  P->d_bhist = (int*)A(sizeof(int) * (size_t)P->ntiles * 2 * P->ctx->nsm);
  P->d_zpart = (double*)A(sizeof(double) * BQ_N * pb->nbins * (size_t)P->nblk_z);
  P->d_zpartc = (int*)A(sizeof(int) * pb->nbins * (size_t)P->nblk_z);
  P->d_bins = (double*)A(sizeof(double) * BQ_N * pb->nbins);
  P->d_binc = (long long*)A(sizeof(long long) * pb->nbins);
  if (!ok) {
    const size_t tot = P->bytes_total;
    delete P;
    return set_error(FKP_ENOMEM, "device allocation failed (plan needs about %.2f GB)", tot / 1e9);
  }
  if (ctx->budget && P->bytes_total > ctx->budget) {
    const size_t tot = P->bytes_total;
    delete P;
    return set_error(FKP_ENOMEM, "plan needs %.2f GB, over the HBM budget", tot / 1e9);
  }
  if (wantB) {
    int rc = bisp_plan_init(P);
    if (rc) { delete P; return rc; }
  }
  CK(cudaMemcpy(P->d_tw, tw.data(), sizeof(float2) * N, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(P->d_lut, lut.data(), sizeof(short) * (n2max + 1), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(P->d_winv, winv.data(), sizeof(float) * 3 * N, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(P->d_hph, hph.data(), sizeof(float2) * N, cudaMemcpyHostToDevice));
  const size_t hbytes = sizeof(double) * (BQ_N * pb->nbins + pb->nbins + DS_COUNT + LAB_NSUM + 8) + 64;
  CK(cudaMallocHost(&P->h_pinned, hbytes));
  for (auto& e : P->ev) CK(cudaEventCreate(&e));
  CK(cudaEventCreateWithFlags(&P->ev_fork, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&P->ev_join, cudaEventDisableTiming));
  CK(cudaStreamCreateWithFlags(&P->side, cudaStreamNonBlocking));
  {
    const int rc = tune_schedule(P);
    if (rc) { delete P; return rc; }
  }
  *out = P;
  return FKP_OK;
}

extern "C" void fkp_plan_destroy(void* plan) {
  auto* P = static_cast<Plan*>(plan);
  if (!P) return;
  cudaSetDevice(P->ctx->device);
  delete P;
}

extern "C" int fkp_plan_sizes(const void* plan, int* nbins, int* ntri, size_t* ws) {
  auto* P = static_cast<const Plan*>(plan);
  if (!P) return set_error(FKP_EINVAL, "NULL plan");
  if (nbins) *nbins = P->pb.nbins;
  if (ntri) *ntri = P->ntri;
  // workspace plus the per-call buffers the plan keeps (tile-sorted and staged
  // catalogs, the fused-batch workspace)
  if (ws) *ws = P->bytes_total + P->sort_cap * (sizeof(float4) + (P->d_vw2 ? sizeof(float) : 0)) +
                P->staging_bytes[0] + P->staging_bytes[1] + P->batch_bytes;
  return FKP_OK;
}

// ----------------------------------------------------------------------------
// catalogs: device views, copying host arrays into plan-owned staging
// ----------------------------------------------------------------------------

int fkp::stage_catalog(Plan* P, const fkp_catalog_t* c, int slot, CatDev& out, cudaStream_t s) {
  if (!c) return set_error(FKP_EINVAL, "NULL catalog");
  if (c->n < 0) return set_error(FKP_EINVAL, "negative catalog size");
  if (c->n > 0 && (!c->x || !c->y || !c->z || !c->nbar))
    return set_error(FKP_EINVAL, "catalog needs x, y, z and nbar (w may be NULL)");
  out.n = c->n;
  if (c->on_device || c->n == 0) {
    out.x = c->x; out.y = c->y; out.z = c->z; out.w = c->w; out.nbar = c->nbar;
    return FKP_OK;
  }
  const size_t need = (size_t)c->n * sizeof(float) * 5;
  if (P->staging_bytes[slot] < need) {
    if (P->staging[slot]) cudaFree(P->staging[slot]);
    P->staging[slot] = nullptr;
    P->staging_bytes[slot] = 0;
    if (cudaMalloc(&P->staging[slot], need) != cudaSuccess)
      return set_error(FKP_ENOMEM, "cannot stage a host catalog of %lld objects", (long long)c->n);
    P->staging_bytes[slot] = need;
  }
  float* base = static_cast<float*>(P->staging[slot]);
  const size_t n = (size_t)c->n;
  const float* src[5] = {c->x, c->y, c->z, c->w, c->nbar};
  const float* dst[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  for (int a = 0; a < 5; ++a) {
    if (!src[a]) continue;
    float* d = base + a * n;
    CK(cudaMemcpyAsync(d, src[a], n * sizeof(float), cudaMemcpyHostToDevice, s));
    dst[a] = d;
  }
  out.x = dst[0]; out.y = dst[1]; out.z = dst[2]; out.w = dst[3]; out.nbar = dst[4];
  return FKP_OK;
}

// ----------------------------------------------------------------------------
// P_l
// ----------------------------------------------------------------------------

// Records a stage event on s.  Inside a stream capture it is recorded as an
// external event, so that the graph keeps it as a timed event node (a plain
// record only orders the captured work).
cudaError_t fkp::record_stage(cudaEvent_t ev, cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  const cudaError_t e = cudaStreamIsCapturing(s, &st);
  if (e != cudaSuccess) return e;
  return st == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal)
                                             : cudaEventRecord(ev, s);
}

// Enqueues scalars and gridding of both catalogs into d_grid (and d_gridw):
// tile counts with the scalar sums, offsets, scatter into tile order, and
// shared-memory accumulation per tile.
// One grid of the pair (which = 1: the interlaced second grid, nodes half a
// cell further; no stage events).
static int grid_pass(Plan* P, const CatDev& gal, const CatDev& ran, cudaStream_t s, int which) {
  const GeomDev& geo = which ? P->g2 : P->g;
  unsigned long long* grid = which ? P->d_grid2 : P->d_grid;
  unsigned long long* gridw = which ? P->d_gridw2 : P->d_gridw;
  const unsigned long long* rgrid = which ? P->rc_grid2 : P->rc_grid;
  const unsigned long long* rgridw = which ? P->rc_gridw2 : P->rc_gridw;
  auto stage = [&](int e) { return which ? cudaSuccess : record_stage(P->ev[e], s); };
  const int N = P->g.N;
  const size_t N3 = (size_t)N * N * N;
  const bool cached = ran.n < 0;  // the plan's cached random grids (fkp_plan_cache_randoms)
  if (cached && !P->rc_valid) return set_error(FKP_ESTATE, "no cached random catalog on this plan");
  const long long ntot = gal.n + (cached ? 0 : ran.n);
  if (ntot >= (1ll << 31)) return set_error(FKP_EINVAL, "at most 2^31-1 objects per call");
  if ((size_t)ntot > P->sort_cap) {
    // a captured graph refers to the old buffers
    if (P->graph_exec) cudaGraphExecDestroy(P->graph_exec);
    P->graph_exec = nullptr;
    bisp_drop_graph(P);
    if (P->d_xyzv) cudaFree(P->d_xyzv);
    if (P->d_vw2) cudaFree(P->d_vw2);
    P->d_xyzv = nullptr;
    P->d_vw2 = nullptr;
    P->sort_cap = 0;
    const size_t cap = (size_t)ntot + ntot / 8 + 1024;
    if (cudaMalloc(&P->d_xyzv, sizeof(float4) * cap) != cudaSuccess)
      return set_error(FKP_ENOMEM, "cannot allocate the tile-sorted catalog (%lld objects)", ntot);
    if (P->d_gridw && cudaMalloc(&P->d_vw2, sizeof(float) * cap) != cudaSuccess)
      return set_error(FKP_ENOMEM, "cannot allocate the tile-sorted catalog (%lld objects)", ntot);
    P->sort_cap = cap;
  }
  // one 1024-thread block per SM for the binning kernels (their shared
  // histogram spans every tile)
  const int nb = P->ctx->nsm;
  auto nblocks = [&](long long n) { return (int)std::max<long long>(1, std::min<long long>(nb, (n + 4095) / 4096)); };
  const int nbg = nblocks(gal.n), nbr = cached ? P->rc_nblk : nblocks(ran.n);
  const long long nran = cached ? P->rc_n : ran.n;
  if (!which) CK(cudaMemsetAsync(P->d_err, 0, sizeof(int) * 4, s));
  CK(stage(0));
  // zero the grids on the side stream while the counts run
  CK(cudaEventRecord(P->ev_fork, s));
  CK(cudaStreamWaitEvent(P->side, P->ev_fork, 0));
  const int ngrid = P->per_object ? P->mt.nfields : 1;  // per object: the moment fields follow F
  CK(cudaMemsetAsync(grid, 0, N3 * 8 * ngrid, P->side));
  if (gridw) CK(cudaMemsetAsync(gridw, 0, N3 * 8, P->side));
  CK(cudaEventRecord(P->ev_join, P->side));
  int* bh_ran = P->d_bhist + (size_t)nbg * P->ntiles;
  CK(launch_bin_count(gal, 0, geo, P->d_scpart, P->d_bhist, P->d_err, nbg, s));
  if (cached)
    CK(cudaMemcpyAsync(P->d_scpart + (size_t)nbg * SC_NSUM, P->rc_part, sizeof(double) * SC_NSUM * nbr,
                       cudaMemcpyDeviceToDevice, s));
  else
    CK(launch_bin_count(ran, 1, geo, P->d_scpart + (size_t)nbg * SC_NSUM, bh_ran, P->d_err, nbr, s));
  CK(launch_scalars_finalize(P->d_scpart, nbg, nbr, gal.n, nran, geo.alpha_mode, P->d_ds, s));
  CK(launch_tile_prefix(P->d_bhist, nbg + (cached ? 0 : nbr), P->ntiles, P->d_tcnt, s));
  CK(launch_scan_tiles(P->d_tcnt, P->ntiles, P->d_toff, P->d_titem, s));
  CK(stage(1));
  CK(cudaStreamWaitEvent(s, P->ev_join, 0));
  const double* obs = P->geom.observer;
  float* vw2 = gridw ? P->d_vw2 : nullptr;
  CK(launch_bin_scatter(gal, 0, geo, obs, P->d_ds, P->d_toff, P->d_bhist, P->d_xyzv, vw2, nullptr, nbg, s));
  if (cached) {
    CK(cudaMemcpyAsync(P->d_ds + DS_COUNT, P->rc_lab, sizeof(double) * LAB_NSUM, cudaMemcpyDeviceToDevice, s));
  } else {
    CK(launch_bin_scatter(ran, 1, geo, obs, P->d_ds, P->d_toff, bh_ran, P->d_xyzv, vw2, P->d_labpart, nbr, s));
    CK(launch_lab_finalize(P->d_labpart, ran.n > 0 ? nbr : 0, P->d_ds + DS_COUNT, s));
  }
  CK(launch_tile_accum(geo, P->d_toff, P->d_titem, gal.n + (cached ? 0 : ran.n), P->d_xyzv, vw2, grid, gridw, s));
  // per-object line of sight: moment field q grids w x^^e[q] with each object's x^
  for (int q = 1; q < ngrid; ++q)
    CK(launch_tile_accum(geo, P->d_toff, P->d_titem, gal.n + ran.n, P->d_xyzv, nullptr, grid + (size_t)q * N3,
                         nullptr, s, P->mt.e[q]));
  if (cached)
    CK(launch_combine_randoms(grid, rgrid, gridw, rgridw, P->d_ds, (long long)N3, P->ctx->nsm, s));
  return FKP_OK;
}

// Enqueues scalars and gridding of both catalogs into d_grid (and d_gridw),
// and for interlaced plans into the second grids too: tile counts with the
// scalar sums, offsets, scatter into tile order, and shared-memory
// accumulation per tile.
int fkp::enqueue_grids(Plan* P, const CatDev& gal, const CatDev& ran, cudaStream_t s) {
  int rc = grid_pass(P, gal, ran, s, 0);
  if (!rc && P->interlace) rc = grid_pass(P, gal, ran, s, 1);
  if (rc) return rc;
  CK(record_stage(P->ev[2], s));
  return FKP_OK;
}

// The randoms' part of the grids without alpha (R = sum_r w W, and R^w =
// sum_r w^2 W for bispectrum plans), the per-block partial scalar sums of
// their count launch and their L^ab sums, kept on the plan for the mocks that
// share this random catalog.
static int cache_randoms(Plan* P, const CatDev& ran, cudaStream_t s) {
  const int N = P->g.N;
  const size_t N3 = (size_t)N * N * N;
  P->rc_valid = false;
  if (P->graph_exec) cudaGraphExecDestroy(P->graph_exec);  // a captured graph may hold the old cache
  P->graph_exec = nullptr;
  P->last_valid = false;
  bisp_drop_graph(P);
  if (ran.n == 0) return FKP_OK;
  if (ran.n >= (1ll << 31)) return set_error(FKP_EINVAL, "at most 2^31-1 randoms");
  const int nb = P->ctx->nsm;
  const int nbr = (int)std::max<long long>(1, std::min<long long>(nb, (ran.n + 4095) / 4096));
  if (!P->rc_grid) {
    P->rc_grid = (unsigned long long*)P->alloc(N3 * 8);
    if (P->d_gridw) P->rc_gridw = (unsigned long long*)P->alloc(N3 * 8);
    if (P->interlace) {
      P->rc_grid2 = (unsigned long long*)P->alloc(N3 * 8);
      if (P->d_gridw) P->rc_gridw2 = (unsigned long long*)P->alloc(N3 * 8);
    }
    P->rc_part = (double*)P->alloc(sizeof(double) * SC_NSUM * nb);
    P->rc_lab = (double*)P->alloc(sizeof(double) * LAB_NSUM);
    if (!P->rc_grid || (P->d_gridw && !P->rc_gridw) || !P->rc_part || !P->rc_lab ||
        (P->interlace && (!P->rc_grid2 || (P->d_gridw && !P->rc_gridw2))))
      return set_error(FKP_ENOMEM, "cannot allocate the cached random grids");
  }
  if ((size_t)ran.n > P->sort_cap) {
    if (P->d_xyzv) cudaFree(P->d_xyzv);
    if (P->d_vw2) cudaFree(P->d_vw2);
    P->d_xyzv = nullptr;
    P->d_vw2 = nullptr;
    P->sort_cap = 0;
    const size_t cap = (size_t)ran.n + ran.n / 8 + 1024;
    if (cudaMalloc(&P->d_xyzv, sizeof(float4) * cap) != cudaSuccess ||
        (P->d_gridw && cudaMalloc(&P->d_vw2, sizeof(float) * cap) != cudaSuccess))
      return set_error(FKP_ENOMEM, "cannot allocate the tile-sorted catalog (%lld objects)", ran.n);
    P->sort_cap = cap;
  }
  float* vw2 = P->d_gridw ? P->d_vw2 : nullptr;
  CK(cudaMemsetAsync(P->d_err, 0, sizeof(int) * 4, s));
  for (int which = 0; which < (P->interlace ? 2 : 1); ++which) {
    const GeomDev& geo = which ? P->g2 : P->g;
    unsigned long long* rg = which ? P->rc_grid2 : P->rc_grid;
    unsigned long long* rgw = which ? P->rc_gridw2 : P->rc_gridw;
    CK(launch_bin_count(ran, 1, geo, P->rc_part, P->d_bhist, P->d_err, nbr, s));
    CK(launch_tile_prefix(P->d_bhist, nbr, P->ntiles, P->d_tcnt, s));
    CK(launch_scan_tiles(P->d_tcnt, P->ntiles, P->d_toff, P->d_titem, s));
    CK(cudaMemsetAsync(rg, 0, N3 * 8, s));
    if (rgw) CK(cudaMemsetAsync(rgw, 0, N3 * 8, s));
    CK(launch_bin_scatter(ran, 1, geo, P->geom.observer, P->d_ds, P->d_toff, P->d_bhist, P->d_xyzv, vw2, P->d_labpart, nbr, s,
                          1));
    CK(launch_lab_finalize(P->d_labpart, nbr, P->rc_lab, s));
    CK(launch_tile_accum(geo, P->d_toff, P->d_titem, ran.n, P->d_xyzv, vw2, rg, rgw, s));
  }
  int herr = 0;
  CK(cudaMemcpyAsync(&herr, P->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (herr)
    return set_error(FKP_EGEOM, "a random lies within assign/2+1 cells of a box face (or is not finite)");
  P->rc_nblk = nbr;
  P->rc_n = ran.n;
  P->rc_valid = true;
  return FKP_OK;
}

extern "C" int fkp_plan_cache_randoms(void* plan, const fkp_catalog_t* ran, void* stream) {
  auto* P = static_cast<Plan*>(plan);
  if (!P || !ran) return set_error(FKP_EINVAL, "NULL plan or catalog");
  if (P->per_object) return set_error(FKP_ESTATE, "FKP_XHAT_OBJECT plans grid the randoms' moments with each mock");
  CK(cudaSetDevice(P->ctx->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CatDev r;
  int rc = stage_catalog(P, ran, 1, r, s);
  if (rc) return rc;
  return cache_randoms(P, r, s);
}

// The random catalog of a call: the given one, or (ran == NULL) the plan's
// cache, marked by n = -1.
int fkp::randoms_of(Plan* P, const fkp_catalog_t* ran, CatDev& r, cudaStream_t s) {
  if (!ran) {
    if (!P->rc_valid) return set_error(FKP_ESTATE, "ran is NULL but the plan has no cached random catalog");
    r = CatDev{};
    r.n = -1;
    return FKP_OK;
  }
  const int rc = stage_catalog(P, ran, 1, r, s);
  if (rc) return rc;
  if (r.n == 0) return set_error(FKP_EINVAL, "the random catalog is empty");
  return FKP_OK;
}

// z-pass parameters of a plan (mode 0: P bins; the bispectrum path sets its
// shell fields on top).
ZParams fkp::zparams(const Plan* P, int mode) {
  ZParams zp{};
  zp.nbins = P->pb.nbins;
  zp.lmax = P->lmax;
  zp.kf = (float)(2.0 * M_PI / P->geom.L);
  zp.lut = P->d_lut;
  zp.winv = P->d_winv;
  zp.mode = mode;
  zp.nshells = 0;
  zp.nsh2 = 0;
  zp.slut = nullptr;
  zp.E = nullptr;
  zp.mm = 0;
  zp.interlace = P->interlace ? 1 : 0;
  zp.hph = P->d_hph;
  zp.scale = P->interlace ? 0.5f : 1.f;
  zp.split68 = (P->want & (FKP_P6B | FKP_P8B)) && P->lmax >= 4 ? 1 : 0;
  return zp;
}

int fkp::enqueue_xy(Plan* P, const unsigned long long* gq, const unsigned long long* gq2, const float* gf,
                    cudaStream_t s, bool events) {
  CK(launch_xpass(gq, gf, P->g, P->mt, P->fp, P->d_tw, P->d_S1, P->ctx->nsm, s, P->sched.x_mult, MockBatch(),
                  P->per_object));
  if (events) CK(record_stage(P->ev[3], s));
  CK(launch_ypass(P->d_S1, gq, gf, P->g, P->mt, P->fp, P->d_tw, P->d_S2, P->d_err + 1, s, P->sched.y_threads));
  if (P->interlace) {
    // the second grid's groups follow the first's; the z-pass applies its
    // half-cell phase e^{-i pi (n_x + n_y + n_z)/N}
    float2* S2b = P->d_S2 + field_elems(P->g.N) * P->mt.ngroups;
    CK(launch_xpass(gq2, nullptr, P->g2, P->mt, P->fp, P->d_tw, P->d_S1, P->ctx->nsm, s, P->sched.x_mult));
    CK(launch_ypass(P->d_S1, gq2, nullptr, P->g2, P->mt, P->fp, P->d_tw, S2b, P->d_err + 1, s, P->sched.y_threads));
  }
  if (events) CK(record_stage(P->ev[4], s));
  return FKP_OK;
}

// Enqueues the three FFT passes, recombination and binning of one base grid
// (of the interlaced pair d_grid, d_grid2 when the plan interlaces).
int fkp::enqueue_fft_bin(Plan* P, const unsigned long long* gq, const float* gf, cudaStream_t s) {
  const int rc = enqueue_xy(P, gq, P->d_grid2, gf, s, true);
  if (rc) return rc;
  const ZParams zp = zparams(P, 0);
  CK(launch_zpass(P->d_S2, P->g, P->mt, P->fp, P->d_tw, zp, P->d_zpart, P->d_zpartc, P->d_err + 1, s,
                  P->ctx->nsm, P->sched.z_threads));
  CK(launch_reduce_bins(P->d_zpart, P->d_zpartc, zpass_blocks(P->g.N, P->sched.z_threads, P->ctx->nsm),
                        P->pb.nbins, P->d_bins, P->d_binc, s));
  CK(record_stage(P->ev[5], s));
  return FKP_OK;
}

// Copies bins and scalars back, synchronizes and fills out.
int fkp::finish_power(Plan* P, cudaStream_t s, fkp_power_out* out, bool have_scalars, double I22u, double N0u) {
  const int nb = P->pb.nbins;
  double* h = static_cast<double*>(P->h_pinned);
  double* hb = h;
  long long* hc = reinterpret_cast<long long*>(h + BQ_N * nb);
  double* hds = h + BQ_N * nb + nb;
  int* herr = reinterpret_cast<int*>(hds + DS_COUNT + LAB_NSUM + 8);
  CK(cudaMemcpyAsync(hb, P->d_bins, sizeof(double) * BQ_N * nb, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(hc, P->d_binc, sizeof(long long) * nb, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(hds, P->d_ds, sizeof(double) * (DS_COUNT + LAB_NSUM), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(herr, P->d_err, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (herr[1] != 0)
    return set_error(FKP_ETIMEOUT, "a bounded device-side wait for a tile copy gave up (flags 0x%x)", herr[1]);
  if (have_scalars && herr[0] != 0)
    return set_error(FKP_EGEOM, "an object lies within assign/2+1 cells of a box face (or is not finite); "
                                "enlarge the box or set periodic=1 (flags 0x%x)", herr[0]);
  if (!out) return FKP_OK;
  double I22 = I22u, N0 = N0u;
  if (have_scalars) {
    out->alpha = hds[DS_ALPHA];
    out->I22 = I22 = hds[DS_I22];
    out->I33 = hds[DS_I33];
    out->N0 = N0 = hds[DS_N0];
    out->N0_fkp = hds[DS_N0FKP];
    out->S3 = hds[DS_S3];
    out->W_g = hds[DS_WG];
    out->W_r = hds[DS_WR];
    out->n_gal = (int64_t)hds[DS_NG];
    out->n_ran = (int64_t)hds[DS_NR];
    for (int a = 0; a < 6; ++a) out->Lab[a] = hds[DS_WR] > 0 ? hds[DS_COUNT + a] / hds[DS_WR] : 0.0;
  } else {
    out->alpha = 0; out->I22 = I22; out->I33 = 0; out->N0 = N0; out->N0_fkp = 0; out->S3 = 0;
    out->W_g = out->W_r = 0; out->n_gal = out->n_ran = 0;
    for (int a = 0; a < 6; ++a) out->Lab[a] = 0;
  }
  for (int b = 0; b < nb; ++b) {
    const double n = (double)hc[b];
    const double s00 = hb[BQ_F00 * nb + b], s20 = hb[BQ_F20 * nb + b], s40 = hb[BQ_F40 * nb + b],
                 s22 = hb[BQ_F22 * nb + b], sk = hb[BQ_K * nb + b];
    const double nan = std::nan("");
    if (out->nmodes) out->nmodes[b] = hc[b];
    if (out->k_eff) out->k_eff[b] = n > 0 ? sk / n : nan;
    if (out->mono_raw) out->mono_raw[b] = n > 0 ? s00 / n / I22 : nan;
    if (out->P0) out->P0[b] = n > 0 ? (s00 / n - N0) / I22 : nan;
    if (out->P2) out->P2[b] = n > 0 && P->lmax >= 2 ? 5.0 * s20 / n / I22 : nan;
    if (out->P4) out->P4[b] = n > 0 && P->lmax >= 4 ? 9.0 * s40 / n / I22 : nan;
    if (out->P4b) out->P4b[b] = n > 0 && P->lmax >= 2 ? (17.5 * s22 - 5.0 * s20 - 3.5 * s00) / n / I22 : nan;
    // split l = 6, 8 (Sec. II.B after eq. P4fast): L_2 L_4 and L_4^2 in Legendre polynomials
    const double s42 = hb[BQ_F42 * nb + b], s44 = hb[BQ_F44 * nb + b];
    const double s60 = 11.0 / 5.0 * (s42 - 2.0 / 7.0 * s20 - 20.0 / 77.0 * s40);
    const double s80 = 1287.0 / 490.0 * (s44 - s00 / 9.0 - 100.0 / 693.0 * s20 - 162.0 / 1001.0 * s40 - 20.0 / 99.0 * s60);
    const bool split = P->lmax >= 4 && (P->want & (FKP_P6B | FKP_P8B));
    if (out->P6b) out->P6b[b] = n > 0 && split ? 13.0 * s60 / n / I22 : nan;
    if (out->P8b) out->P8b[b] = n > 0 && split ? 17.0 * s80 / n / I22 : nan;
  }
  float t = 0.f;
  for (int i = 0; i < 8; ++i) out->timing_ms[i] = 0.f;
  out->graph = 0;
  if (cudaEventElapsedTime(&t, P->ev[0], P->ev[1]) == cudaSuccess) out->timing_ms[0] = t;
  if (cudaEventElapsedTime(&t, P->ev[1], P->ev[2]) == cudaSuccess) out->timing_ms[1] = t;
  if (cudaEventElapsedTime(&t, P->ev[2], P->ev[3]) == cudaSuccess) out->timing_ms[2] = t;
  if (cudaEventElapsedTime(&t, P->ev[3], P->ev[4]) == cudaSuccess) out->timing_ms[3] = t;
  if (cudaEventElapsedTime(&t, P->ev[4], P->ev[5]) == cudaSuccess) out->timing_ms[4] = t;
  if (cudaEventElapsedTime(&t, P->ev[0], P->ev[5]) == cudaSuccess) out->timing_ms[7] = t;
  cudaGetLastError();  // events not recorded on this path leave a benign error
  return FKP_OK;
}

static bool same_cat(const CatDev& a, const CatDev& b) { return std::memcmp(&a, &b, sizeof(CatDev)) == 0; }

// Captures gridding + FFT passes + binning of these catalogs into the plan's
// graph, on the plan's own stream (the legacy default stream cannot capture).
static int capture_power(Plan* P, const CatDev& g, const CatDev& r) {
  if (!P->cap_stream) CK(cudaStreamCreateWithFlags(&P->cap_stream, cudaStreamNonBlocking));
  if (P->graph_exec) cudaGraphExecDestroy(P->graph_exec);
  P->graph_exec = nullptr;
  CK(cudaStreamBeginCapture(P->cap_stream, cudaStreamCaptureModeThreadLocal));
  int rc = enqueue_grids(P, g, r, P->cap_stream);
  if (!rc) rc = enqueue_fft_bin(P, P->d_grid, nullptr, P->cap_stream);
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(P->cap_stream, &graph);
  if (rc || e != cudaSuccess || !graph) {
    if (graph) cudaGraphDestroy(graph);
    return rc ? rc : set_error(FKP_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
  }
  const cudaError_t ei = cudaGraphInstantiate(&P->graph_exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) {
    P->graph_exec = nullptr;
    return set_error(FKP_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(ei));
  }
  P->graph_key[0] = g;
  P->graph_key[1] = r;
  return FKP_OK;
}

// Enqueues the device part of one power call: the plan's graph when the
// catalogs are those it was captured with; a new capture on the second
// identical call in a row; plain launches otherwise.  *replayed tells which.
static int enqueue_power(Plan* P, const CatDev& g, const CatDev& r, bool device_cats, cudaStream_t s,
                         int* replayed) {
  *replayed = 0;
  if (P->graphs && device_cats) {
    const bool cached = P->graph_exec && same_cat(g, P->graph_key[0]) && same_cat(r, P->graph_key[1]);
    if (!cached && P->last_valid && same_cat(g, P->last_key[0]) && same_cat(r, P->last_key[1])) {
      if (capture_power(P, g, r) != FKP_OK) {
        cudaGetLastError();
        P->graphs = false;  // plain launches from now on
      }
    }
    if (P->graphs && P->graph_exec && same_cat(g, P->graph_key[0]) && same_cat(r, P->graph_key[1])) {
      CK(cudaGraphLaunch(P->graph_exec, s));
      ++P->graph_launches;
      *replayed = 1;
      return FKP_OK;
    }
    P->last_key[0] = g;
    P->last_key[1] = r;
    P->last_valid = true;
  }
  int rc = enqueue_grids(P, g, r, s);
  if (rc) return rc;
  return enqueue_fft_bin(P, P->d_grid, nullptr, s);
}

extern "C" int fkp_plan_set_graphs(void* plan, int enable) {
  auto* P = static_cast<Plan*>(plan);
  if (!P) return set_error(FKP_EINVAL, "NULL plan");
  P->graphs = enable != 0;
  if (!P->graphs && P->graph_exec) {
    cudaGraphExecDestroy(P->graph_exec);
    P->graph_exec = nullptr;
  }
  if (!P->graphs) bisp_drop_graph(P);
  P->last_valid = false;
  return FKP_OK;
}

extern "C" int fkp_power(void* plan, const fkp_catalog_t* gal, const fkp_catalog_t* ran, void* stream,
                         fkp_power_out* out) {
  auto* P = static_cast<Plan*>(plan);
  if (!P) return set_error(FKP_EINVAL, "NULL plan");
  CK(cudaSetDevice(P->ctx->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CatDev g, r;
  int rc = stage_catalog(P, gal, 0, g, s);
  if (rc) return rc;
  rc = randoms_of(P, ran, r, s);
  if (rc) return rc;
  const bool device_cats = (gal->on_device || gal->n == 0) && (!ran || ran->on_device || ran->n == 0);
  int replayed = 0;
  rc = enqueue_power(P, g, r, device_cats, s, &replayed);
  if (rc) return rc;
  rc = finish_power(P, s, out, true, 0, 0);
  if (out) out->graph = replayed;
  return rc;
}

extern "C" int fkp_grid(void* plan, const fkp_catalog_t* gal, const fkp_catalog_t* ran, int which, long long* F,
                        long long* Fw, void* stream) {
  auto* P = static_cast<Plan*>(plan);
  if (!P || !gal || !F) return set_error(FKP_EINVAL, "NULL plan, catalog or output");
  if (which != 0 && !(which == 1 && P->interlace))
    return set_error(FKP_EINVAL, "which = %d: 0, or 1 for the second grid of an interlaced plan", which);
  if (Fw && !P->d_gridw) return set_error(FKP_EINVAL, "the plan keeps no F^w grid (no bispectrum outputs)");
  CK(cudaSetDevice(P->ctx->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CatDev g, r;
  int rc = stage_catalog(P, gal, 0, g, s);
  if (rc) return rc;
  rc = randoms_of(P, ran, r, s);
  if (rc) return rc;
  rc = enqueue_grids(P, g, r, s);
  if (rc) return rc;
  const size_t N = (size_t)P->g.N, bytes = N * N * N * sizeof(long long);
  CK(cudaMemcpyAsync(F, which ? P->d_grid2 : P->d_grid, bytes, cudaMemcpyDefault, s));
  if (Fw) CK(cudaMemcpyAsync(Fw, which ? P->d_gridw2 : P->d_gridw, bytes, cudaMemcpyDefault, s));
  int* herr = reinterpret_cast<int*>(P->h_pinned);
  CK(cudaMemcpyAsync(herr, P->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (herr[0] != 0)
    return set_error(FKP_EGEOM, "an object lies within assign/2+1 cells of a box face (or is not finite); "
                                "enlarge the box or set periodic=1 (flags 0x%x)", herr[0]);
  return FKP_OK;
}

// Per-mock element counts of the fused batch workspace.
namespace {
struct BatchSizes {
  size_t grid, s1, s2, zpart, zpartc, bins, binc, ds, err;
};
BatchSizes batch_sizes(const fkp::Plan* P) {
  const size_t N = (size_t)P->g.N, half = fkp::field_elems(P->g.N);
  BatchSizes z;
  z.grid = N * N * N;
  z.s1 = half * P->mt.nfields;
  z.s2 = half * P->mt.ngroups;
  z.zpart = (size_t)BQ_N * P->pb.nbins * P->nblk_z;
  z.zpartc = (size_t)P->pb.nbins * P->nblk_z;
  z.bins = (size_t)BQ_N * P->pb.nbins;
  z.binc = (size_t)P->pb.nbins;
  z.ds = DS_COUNT + LAB_NSUM + 8;
  z.err = 4;
  return z;
}
size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }
}  // namespace

// Sizes (and on request allocates) the fused batch workspace for nmock mocks.
static int reserve_batch(fkp::Plan* P, int nmock) {
  using namespace fkp;
  if (P->batch_cap >= nmock) return FKP_OK;
  const BatchSizes z = batch_sizes(P);
  const size_t K = (size_t)nmock;
  const size_t parts[9] = {align256(K * z.grid * 8),  align256(K * z.s1 * 8),     align256(K * z.s2 * 8),
                           align256(K * z.zpart * 8), align256(K * z.zpartc * 4), align256(K * z.bins * 8),
                           align256(K * z.binc * 8),  align256(K * z.ds * 8),     align256(K * z.err * 4)};
  size_t tot = 0;
  for (size_t b : parts) tot += b;
  if (P->ctx->budget && P->bytes_total + tot > P->ctx->budget)
    return set_error(FKP_ENOMEM, "a batch of %d mocks needs %.2f GB beyond the plan's %.2f GB, over the HBM budget",
                     nmock, tot / 1e9, P->bytes_total / 1e9);
  if (P->batch_mem) cudaFree(P->batch_mem);
  P->batch_mem = nullptr;
  P->batch_cap = 0;
  P->batch_bytes = 0;
  if (cudaMalloc(&P->batch_mem, tot) != cudaSuccess) {
    cudaGetLastError();
    P->batch_mem = nullptr;
    return set_error(FKP_ENOMEM, "cannot allocate %.2f GB for a batch of %d mocks", tot / 1e9, nmock);
  }
  char* m = static_cast<char*>(P->batch_mem);
  P->b_grid = reinterpret_cast<unsigned long long*>(m);  m += parts[0];
  P->b_S1 = reinterpret_cast<float2*>(m);                m += parts[1];
  P->b_S2 = reinterpret_cast<float2*>(m);                m += parts[2];
  P->b_zpart = reinterpret_cast<double*>(m);             m += parts[3];
  P->b_zpartc = reinterpret_cast<int*>(m);               m += parts[4];
  P->b_bins = reinterpret_cast<double*>(m);              m += parts[5];
  P->b_binc = reinterpret_cast<long long*>(m);           m += parts[6];
  P->b_ds = reinterpret_cast<double*>(m);                m += parts[7];
  P->b_err = reinterpret_cast<int*>(m);
  P->batch_cap = nmock;
  P->batch_bytes = tot;
  return FKP_OK;
}

extern "C" int fkp_power_batch(void* plan, int nmock, const fkp_catalog_t* gals, const fkp_catalog_t* rans,
                               void* stream, fkp_power_out* outs) {
  auto* P = static_cast<Plan*>(plan);
  if (!P) return set_error(FKP_EINVAL, "NULL plan");
  if (nmock < 1 || nmock > 65535) return set_error(FKP_EINVAL, "nmock = %d (1 .. 65535)", nmock);
  if (P->interlace) return set_error(FKP_EINVAL, "the fused batch does not interlace: use fkp_power per mock");
  if (P->per_object) return set_error(FKP_ESTATE, "the fused batch forms the moments at the nodes: use fkp_power");
  if (!gals) return set_error(FKP_EINVAL, "NULL catalog array");
  if (!rans && !P->rc_valid) return set_error(FKP_ESTATE, "rans is NULL but the plan has no cached random catalog");
  CK(cudaSetDevice(P->ctx->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc = reserve_batch(P, nmock);
  if (rc) return rc;
  const BatchSizes z = batch_sizes(P);
  // gridding, mock by mock (each launch shaped by its own catalogs), into the
  // mock's grid, scalars and flags
  unsigned long long* const grid0 = P->d_grid;
  double* const ds0 = P->d_ds;
  int* const err0 = P->d_err;
  CK(cudaEventRecord(P->ev[9], s));
  for (int k = 0; k < nmock; ++k) {
    CatDev g, r;
    rc = stage_catalog(P, &gals[k], 0, g, s);
    if (!rc) rc = randoms_of(P, rans ? &rans[k] : nullptr, r, s);
    if (rc) return rc;
    P->d_grid = P->b_grid + k * z.grid;
    P->d_ds = P->b_ds + k * z.ds;
    P->d_err = P->b_err + k * z.err;
    rc = enqueue_grids(P, g, r, s);
    P->d_grid = grid0;
    P->d_ds = ds0;
    P->d_err = err0;
    if (rc) return rc;
  }
  // the three FFT passes and the bin reduction: one launch each for all mocks
  // (blockIdx.z / blockIdx.y = mock); bounded-wait flags go to mock 0's word
  int* perr = P->b_err + 1;
  MockBatch mx;
  mx.n = nmock; mx.in = (long long)z.grid; mx.out = (long long)z.s1;
  CK(launch_xpass(P->b_grid, nullptr, P->g, P->mt, P->fp, P->d_tw, P->b_S1, P->ctx->nsm, s, P->sched.x_mult, mx));
  CK(cudaEventRecord(P->ev[3], s));
  MockBatch my;
  my.n = nmock; my.in = (long long)z.s1; my.in2 = (long long)z.grid; my.out = (long long)z.s2;
  CK(launch_ypass(P->b_S1, P->b_grid, nullptr, P->g, P->mt, P->fp, P->d_tw, P->b_S2, perr, s, P->sched.y_threads,
                  my));
  CK(cudaEventRecord(P->ev[4], s));
  const ZParams zp = zparams(P, 0);
  MockBatch mz;
  mz.n = nmock; mz.in = (long long)z.s2; mz.out = (long long)z.zpart; mz.out2 = (long long)z.zpartc;
  CK(launch_zpass(P->b_S2, P->g, P->mt, P->fp, P->d_tw, zp, P->b_zpart, P->b_zpartc, perr, s, P->ctx->nsm,
                  P->sched.z_threads, mz));
  CK(launch_reduce_bins(P->b_zpart, P->b_zpartc, zpass_blocks(P->g.N, P->sched.z_threads, P->ctx->nsm), P->pb.nbins,
                        P->b_bins, P->b_binc, s, nmock, (long long)z.zpart, (long long)z.zpartc));
  CK(cudaEventRecord(P->ev[5], s));
  // bins and scalars back, mock by mock
  double* const bins0 = P->d_bins;
  long long* const binc0 = P->d_binc;
  float tg = 0.f, tx = 0.f, ty = 0.f, tz = 0.f, tt = 0.f;
  for (int k = 0; k < nmock; ++k) {
    P->d_bins = P->b_bins + k * z.bins;
    P->d_binc = P->b_binc + k * z.binc;
    P->d_ds = P->b_ds + k * z.ds;
    P->d_err = P->b_err + k * z.err;
    rc = finish_power(P, s, outs ? &outs[k] : nullptr, true, 0, 0);
    P->d_bins = bins0;
    P->d_binc = binc0;
    P->d_ds = ds0;
    P->d_err = err0;
    if (rc) return rc;
    if (k == 0) {
      cudaEventElapsedTime(&tg, P->ev[9], P->ev[2]);
      cudaEventElapsedTime(&tx, P->ev[2], P->ev[3]);
      cudaEventElapsedTime(&ty, P->ev[3], P->ev[4]);
      cudaEventElapsedTime(&tz, P->ev[4], P->ev[5]);
      cudaEventElapsedTime(&tt, P->ev[9], P->ev[5]);
      cudaGetLastError();
    }
    if (outs) {
      // stage times of the whole batch
      float* t = outs[k].timing_ms;
      t[0] = 0.f; t[1] = tg; t[2] = tx; t[3] = ty; t[4] = tz; t[5] = t[6] = 0.f; t[7] = tt;
      outs[k].graph = 0;
    }
  }
  return FKP_OK;
}

extern "C" int fkp_selftest_bounded_wait(int device, unsigned polls) {
  if (polls < 1 || polls > kWaitLimit) return set_error(FKP_EINVAL, "polls must be in 1 .. %u", kWaitLimit);
  int ndev = 0;
  CK(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return set_error(FKP_EINVAL, "bad device %d", device);
  CK(cudaSetDevice(device));
  int* d_flag = nullptr;
  int h_flag = 0;
  CK(cudaMalloc(&d_flag, sizeof(int)));
  cudaError_t e = cudaMemset(d_flag, 0, sizeof(int));
  if (e == cudaSuccess) e = launch_wait_selftest(polls, d_flag, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(&h_flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d_flag);
  if (e != cudaSuccess) return set_error(FKP_ECUDA, "bounded-wait self-test: %s", cudaGetErrorString(e));
  if (h_flag == 1)
    return set_error(FKP_ETIMEOUT, "the bounded wait gave up after %u polls on a barrier nothing arrives at", polls);
  return set_error(FKP_ESTATE, "bounded-wait self-test: unexpected flag %d", h_flag);
}

extern "C" int fkp_power_from_grid(void* plan, const float* F, double I22, double N0, void* stream,
                                   fkp_power_out* out) {
  auto* P = static_cast<Plan*>(plan);
  if (!P || !F) return set_error(FKP_EINVAL, "NULL plan or grid");
  if (P->interlace) return set_error(FKP_EINVAL, "a given field has no interlaced partner: use a plan without interlace");
  if (P->per_object) return set_error(FKP_ESTATE, "a given field has no objects to take x^ from (FKP_XHAT_OBJECT)");
  CK(cudaSetDevice(P->ctx->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CK(cudaMemsetAsync(P->d_err, 0, sizeof(int) * 4, s));
  CK(cudaEventRecord(P->ev[0], s));
  CK(cudaEventRecord(P->ev[1], s));
  CK(cudaEventRecord(P->ev[2], s));
  int rc = enqueue_fft_bin(P, nullptr, F, s);
  if (rc) return rc;
  return finish_power(P, s, out, false, I22, N0);
}
