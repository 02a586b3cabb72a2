// Host runtime of the C ABI declared in include/wslda_td.h.
//
// A context owns boxes; a box owns D + 2 state buffers (phi, the slot for the
// next f_{k-1} and D history values: five for AB4AM5, Alg. 2), the site
// fields and the chunked density partials. A step is, per box, on the
// context's stream (or a forked one when boxes are batched):
//   stage X (f, predictor, corrector partial) + norm finalise -> phi_p, c, f_{k-1}
//   densities(phi_p) + potentials [+ friction terms]          -> W, D
//   stage Y (f(phi_p), corrector completion) + norm finalise  -> phi_k
//   densities(phi_k) + potentials [+ friction terms]          -> W, D
// followed by a pointer rotation of the history slots (Alg. 2 steps 5-7).
// The static solver (scf.cu), the uniform seed (uniform.cu), the allocation-
// free density call (noalloc.cu) and the network kernels (convnet.cu) have
// their own files.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/wslda_td.h"
#include "internal.cuh"

namespace wslda {
std::vector<KernelSet>& registry() {
  static std::vector<KernelSet> r;
  return r;
}
}  // namespace wslda

using namespace wslda;

namespace {

enum { PROF_X = 0, PROF_Y = 1, PROF_DENS = 2, PROF_POT = 3, PROF_AUX = 4, NPROF = 5 };

struct Box {
  wslda_lattice lat{};
  wslda_functional fn{};
  FunctionalDev fdev{};
  int64_t n = 0;
  int M = 0;
  const KernelSet* ks = nullptr;
  int ncl = 0;           // persistent stage launches: clusters (0 = one cluster per state)
  const KernelSet* ks_y = nullptr;  // launch variant of the corrector stage (NULL: ks)
  int ncl_y = 0;
  int kt[3] = {1, 1, 1};  // lanes per x / y / z pencil the kinetic tables are ordered for
  size_t csize = 0;      // bytes per complex element (8 or 16)
  int D = 3;             // history values the predictor reads (AB3AM4 2, AB4AM5 3, AB5AM5 4)
  void* slot[6] = {};    // D + 2 state buffers [n][2][M]
  int iphi = 0, ih[5] = {1, 2, 3, 4, 5};  // ih[0]: next f_{k-1}; ih[1..D]: f_{k-2}, ..., f_{k-1-D}
  double *vext = nullptr, *dext = nullptr, *lam = nullptr, *rho = nullptr, *nu = nullptr, *U = nullptr,
         *delta = nullptr;
  void* WD = nullptr;                   // working-precision H fields {W, Re D, Im D, 0}
  double* sc[6] = {};                   // per-slot per-state scale (deferred normalisation)
  void *ktab = nullptr, *tw = nullptr;  // per-axis kinetic symbol and twiddles
  double *wm = nullptr, *wp = nullptr;  // double weights
  void *wm_r = nullptr, *wp_r = nullptr;
  double* part = nullptr;
  int nchunk = 1;
  int64_t chunk = 1;
  double* Ebuf = nullptr;
  double* npart = nullptr;  // [n][16] per-CTA norm partials
  double* ekin2 = nullptr;
  double* out8 = nullptr;
  double e0 = 0.0, n0 = 0.0;  // E_tot - mu N and N of the states at wslda_start
  // quantum friction (Sec. 5.2.4): coefficients, scratch state buffer, fields
  bool fric = false;
  double f_alpha = 0.0, f_beta = 0.0, f_gamma = 0.0, f_rho0 = 1.0, f_nreq = 1.0;
  void* f_scratch = nullptr;
  double *f_div = nullptr, *f_bp = nullptr;
  // current terms (functional with A != 1): per-state scratch [n][2][M] (the
  // per-state contributions to j, then the current term of H phi), {tau, j}
  // [4][M], current potential {A_x, A_y, A_z, div A / 2} [M], <H>_n partials
  // [n][16], per-axis first-derivative columns
  bool cur = false;
  void* cur_buf = nullptr;
  double* tauj = nullptr;
  void* av = nullptr;
  double* ecur = nullptr;
  double* d1 = nullptr;
  // spin-imbalanced ASLDA: the second species' densities {tau, j}, rho, V,
  // current potential; the alpha fields {alpha_a/2, alpha_b/2}; the first
  // columns of the Eq. D2 matrices; per-site scratch of the potentials; the
  // v-part density partials; zero weights (double and working precision)
  bool aslda = false;
  double mu_b = 0.0;
  double *tauj_b = nullptr, *rho_b = nullptr, *U_b = nullptr, *d2 = nullptr, *af = nullptr, *part_b = nullptr;
  void *av_b = nullptr, *alf = nullptr;
  double* wzero = nullptr;
  void* wzero_r = nullptr;
  bool loaded = false;
  void* ptr(int i) const { return slot[i]; }
};

}  // namespace

struct wslda_ctx {
  int prec = 0;
  int scheme_depth = 3;           // history depth of the integrator of boxes added from now on
  cudaStream_t stream = nullptr;  // the caller's stream
  cudaStream_t cur = nullptr;     // stream the box-level launches go to (stream, or a forked one)
  // batched execution: boxes spread over forked streams, four steps captured
  // in one CUDA graph per history-slot phase (the rotation has period 4)
  bool use_graph = false;
  std::vector<cudaStream_t> side;
  cudaEvent_t fork_ev = nullptr;
  std::vector<cudaEvent_t> join_ev;
  std::vector<std::pair<std::vector<int>, cudaGraphExec_t>> graphs;
  std::vector<int64_t> graph_kernels;  // kernels per graph (launch accounting)
  double graph_dt = 0.0;
  cudaStream_t cap = nullptr;      // context-owned stream the graphs are captured and replayed on
  cudaEvent_t cap_in = nullptr, cap_out = nullptr;
  std::vector<Box> boxes;
  std::string err;
  int status = WSLDA_OK;
  int* err_d = nullptr;
  double t = 0.0;
  int64_t steps = 0;
  bool started = false;
  double dt_start = 0.0;
  int64_t bytes = 0;
  std::vector<void*> allocs;
  bool prof = false;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
  std::vector<cudaEvent_t> evpool;
  double prof_ms[NPROF] = {};
  int64_t prof_n[NPROF] = {};
  int64_t launches = 0;  // kernels this context has launched
};

namespace {

wslda_status fail(wslda_ctx* c, wslda_status st, const std::string& msg) {
  if (c && c->status == WSLDA_OK) {
    c->status = st;
    c->err = msg;
  }
  return st;
}

#define CUDA_TRY(ctx, call)                                                                              \
  do {                                                                                                   \
    cudaError_t e_ = (call);                                                                             \
    if (e_ != cudaSuccess)                                                                               \
      return fail(ctx, WSLDA_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));                 \
  } while (0)

#define CUDA_TRY_NEG(ctx, call)                                                                          \
  do {                                                                                                   \
    cudaError_t e_ = (call);                                                                             \
    if (e_ != cudaSuccess)                                                                               \
      return -fail(ctx, WSLDA_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));                \
  } while (0)

#define CHECK_CTX(ctx)                                                           \
  do {                                                                           \
    if (!(ctx)) return WSLDA_EINVAL;                                             \
    if ((ctx)->status != WSLDA_OK) return WSLDA_ESTATE;                          \
  } while (0)

cudaError_t dalloc(wslda_ctx* c, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
  if (e == cudaSuccess) {
    c->allocs.push_back(*p);
    c->bytes += int64_t(bytes);
  }
  return e;
}

std::vector<const KernelSet*> find_variants(int prec, int nx, int ny, int nz) {
  std::vector<const KernelSet*> v;
  for (const KernelSet& k : registry())
    if (k.prec == prec && k.nx == nx && k.ny == ny && k.nz == nz) v.push_back(&k);
  return v;
}

const KernelSet* find_kernels(int prec, int nx, int ny, int nz) {
  std::vector<const KernelSet*> v = find_variants(prec, nx, ny, nz);
  if (v.empty()) return nullptr;
  const char* env = getenv("WSLDA_VARIANT");
  if (env) {
    const int i = atoi(env);
    if (i >= 0 && i < int(v.size())) return v[i];
  }
  return v[0];
}

int resident_clusters(const KernelSet* ks) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ks->cs * 16);
  cfg.blockDim = dim3(ks->bt);
  cfg.dynamicSmemBytes = ks->smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = ks->cs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  for (int m = 0; m < NMODES; ++m) {
    cudaFuncSetAttribute(ks->fn[m], cudaFuncAttributeMaxDynamicSharedMemorySize, int(ks->smem));
    if (ks->cs > 8) cudaFuncSetAttribute(ks->fn[m], cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  }
  int ncl = 0;
  if (cudaOccupancyMaxActiveClusters(&ncl, ks->fn[MODE_X], &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return ncl;
}

int brev_host(int j, int T) {
  int r = 0;
  for (int b = 1; b < T; b <<= 1) {
    r <<= 1;
    if (j & b) r |= 1;
  }
  return r;
}

// Kinetic symbol per slot along one axis: slot s = j + T m holds frequency
// m + N1 brev(j) after the forward pencil transform (identity for T = 1).
void axis_tables(int N, int T, double d, double scale, std::vector<double>& k2, std::vector<double>& k1,
                 std::vector<double>& twr, std::vector<double>& twi) {
  const int N1 = N / T;
  const long double L = (long double)N * d;
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int s = 0; s < N; ++s) {
    const int j = s % T, m = s / T;
    const int f = m + N1 * brev_host(j, T);
    const long double k = (f < N / 2) ? 2 * pi * f / L : 2 * pi * (f - N) / L;
    k2.push_back(double(k * k) * scale);
    // first derivative symbol k / M, the Nyquist mode zeroed (Eq. derivative-spectral, odd r)
    k1.push_back(f == N / 2 ? 0.0 : double(k) * 2.0 * scale);
    twr.push_back(double(cosl(2 * pi * s / N)));
    twi.push_back(double(-sinl(2 * pi * s / N)));
  }
}

double default_cutoff(const wslda_lattice& l) {
  return 0.5 * M_PI * M_PI * (1.0 / (l.dx * l.dx) + 1.0 / (l.dy * l.dy) + 1.0 / (l.dz * l.dz));
}

cudaEvent_t take_event(wslda_ctx* c) {
  if (!c->evpool.empty()) {
    cudaEvent_t e = c->evpool.back();
    c->evpool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

struct ProfScope {
  wslda_ctx* c;
  int kind;
  cudaEvent_t a = nullptr, b = nullptr;
  ProfScope(wslda_ctx* c_, int k) : c(c_), kind(k) {
    if (c->prof) {
      a = take_event(c);
      b = take_event(c);
      cudaEventRecord(a, c->cur);
    }
  }
  ~ProfScope() {
    if (c->prof) {
      cudaEventRecord(b, c->cur);
      c->pending.push_back({kind, {a, b}});
    }
  }
};

void collect_profile(wslda_ctx* c) {
  if (c->pending.empty()) return;
  cudaStreamSynchronize(c->stream);
  for (auto& p : c->pending) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p.second.first, p.second.second);
    c->prof_ms[p.first] += ms;
    c->prof_n[p.first] += 1;
    c->evpool.push_back(p.second.first);
    c->evpool.push_back(p.second.second);
  }
  c->pending.clear();
}

template <typename R>
StageArgs<R> base_args(const Box& b, double dV) {
  StageArgs<R> a = {};
  a.WD = static_cast<const fx4<R>*>(b.WD);
  a.ktab = static_cast<const R*>(b.ktab);
  a.tw = static_cast<const cx<R>*>(b.tw);
  a.E = b.Ebuf;
  a.npart = b.npart;
  a.out2 = b.ekin2;
  a.dV = dV;
  a.ycoef = b.D == 2 ? 9.0 / 24.0 : 251.0 / 720.0;  // new term of Eq. AM4 / Eq. AM5
  a.nstates = int(b.n);
  return a;
}

double box_dV(const Box& b) { return b.lat.dx * b.lat.dy * b.lat.dz; }

// predictor-stage kernel mode of the box's scheme
int x_mode(const Box& b) { return b.D == 2 ? MODE_X3 : (b.D == 4 ? MODE_X5 : MODE_X); }

// whether a launch variant reads the box's kinetic tables in their order
bool same_layout(const KernelSet* k, const Box& b) { return k->tx == b.kt[0] && k->ty == b.kt[1] && k->tz == b.kt[2]; }

// A stage launch; normalising modes are followed by the kernel that turns the
// per-CTA norm partials into the per-state factor (same profiling scope).
template <typename R>
wslda_status launch_mode(wslda_ctx* c, Box& b, int mode, StageArgs<R>& a, int kind) {
  a.err = c->err_d;
  if (b.n == 0) return WSLDA_OK;
  const bool ym = mode == MODE_Y && b.ks_y;
  const KernelSet* ks = ym ? b.ks_y : b.ks;
  if (!same_layout(ks, b)) return fail(c, WSLDA_EUNSUPPORTED, "launch variant does not match the kinetic tables");
  const bool gen = b.cur && applies_h(mode);
  if (gen) {
    // current term -(i/2){A, grad} phi of this launch's input states and its
    // part of <H>_n, read by the stage below. It runs on the stage's own launch
    // variant: its <H>_n partials are per CTA of that variant's clusters.
    // Spin-imbalanced ASLDA: each row its own current potential, then the
    // transformed alpha phi parts of Eq. kinop-alpha added to the same buffer.
    ProfScope pg(c, PROF_AUX);
    StageArgs<R> g = base_args<R>(b, box_dV(b));
    g.phi = a.phi;
    g.sc_in = a.sc_in;
    g.h0 = static_cast<cx<R>*>(b.cur_buf);
    g.av = static_cast<const fx4<R>*>(b.av);
    g.av2 = static_cast<const fx4<R>*>(b.av_b);
    g.alf = static_cast<const cx<R>*>(b.alf);
    g.ecur = b.ecur;
    g.err = c->err_d;
    CUDA_TRY(c, ks->launch[MODE_AGRAD](&g, int(b.n), 0, c->cur));
    c->launches += 1;
    if (b.aslda) {
      CUDA_TRY(c, ks->launch[MODE_KALPHA](&g, int(b.n), 0, c->cur));
      c->launches += 1;
    }
    a.cur = static_cast<const cx<R>*>(b.cur_buf);
    a.ecur = b.ecur;
    a.alf = static_cast<const cx<R>*>(b.alf);
  }
  ProfScope ps(c, kind);
  if (gen) CUDA_TRY(c, ks->launch_gen[mode](&a, int(b.n), 0, c->cur));
  else CUDA_TRY(c, ks->launch[mode](&a, int(b.n), ym ? b.ncl_y : b.ncl, c->cur));
  c->launches += 1;
  const bool norm_out = mode == MODE_X || mode == MODE_X3 || mode == MODE_X5 || mode == MODE_Y ||
                        (mode == MODE_HORNER && a.normalize);
  if (norm_out) {
    CUDA_TRY(c, launch_finalize_norm(a.npart, ks->cs, b.n, box_dV(b), a.sc_out, c->err_d, c->cur));
    c->launches += 1;
  }
  return WSLDA_OK;
}

// densities of slot `islot` -> potentials -> H fields
// Spin-imbalanced ASLDA: {tau, j} and the density partials of the u part
// (weights 0, f(E)) and of the v part (f(-E), 0), then the potentials and the
// fields of H.
template <typename R>
wslda_status refresh_aslda(wslda_ctx* c, Box& b, int islot, int init_lam) {
  const double* wsets[2][2] = {{b.wzero, b.wp}, {b.wm, b.wzero}};
  const void* rsets[2][2] = {{b.wzero_r, b.wp_r}, {b.wm_r, b.wzero_r}};
  double* tj[2] = {b.tauj, b.tauj_b};
  double* parts[2] = {b.part, b.part_b};
  for (int sp = 0; sp < 2; ++sp) {
    if (b.n > 0) {
      StageArgs<R> a = base_args<R>(b, box_dV(b));
      a.phi = static_cast<cx<R>*>(b.ptr(islot));
      a.h0 = static_cast<cx<R>*>(b.cur_buf);
      a.sc_in = b.sc[islot];
      a.wm = wsets[sp][0];
      a.wp = wsets[sp][1];
      wslda_status st = launch_mode<R>(c, b, MODE_GRAD, a, PROF_DENS);
      if (st) return st;
      ProfScope pj(c, PROF_DENS);
      c->launches += 3;
      // the v-part partial buffer is the scratch of the sum (the u-part partials are kept)
      CUDA_TRY(c, launch_sum_tauj<R>(static_cast<const cx<R>*>(b.cur_buf), b.n, b.M, b.nchunk, b.chunk, b.part_b,
                                     tj[sp], tj[sp] + b.M, c->cur));
      CUDA_TRY(c, launch_density_partial<R>(static_cast<const cx<R>*>(b.ptr(islot)), b.sc[islot],
                                            static_cast<const R*>(rsets[sp][0]), static_cast<const R*>(rsets[sp][1]),
                                            b.n, b.M, b.nchunk, b.chunk, parts[sp], c->cur));
    } else {
      CUDA_TRY(c, cudaMemsetAsync(tj[sp], 0, size_t(4) * b.M * 8, c->cur));
      CUDA_TRY(c, cudaMemsetAsync(parts[sp], 0, size_t(3) * b.M * b.nchunk * sizeof(double), c->cur));
    }
  }
  ProfScope ps2(c, PROF_POT);
  c->launches += 2;
  CUDA_TRY(c, launch_aslda_potentials(b.part, b.part_b, b.nchunk, b.M, b.tauj, b.tauj_b, b.vext, b.fdev.mu, b.mu_b,
                                      b.fdev.C, b.fdev.ec, b.fdev.rho_floor, b.lam, init_lam, b.rho, b.rho_b, b.nu,
                                      b.U, b.U_b, b.delta, b.af, c->cur));
  CUDA_TRY(c, launch_aslda_fields<R>(b.lat.nx, b.lat.ny, b.lat.nz, b.af, b.U, b.U_b, b.delta, b.vext, b.dext,
                                     b.fdev.mu, b.mu_b, b.d1, b.d2, static_cast<fx4<R>*>(b.WD),
                                     static_cast<cx<R>*>(b.alf), static_cast<fx4<R>*>(b.av),
                                     static_cast<fx4<R>*>(b.av_b), c->cur));
  return WSLDA_OK;
}

template <typename R>
wslda_status refresh_fields_t(wslda_ctx* c, Box& b, int islot, int init_lam) {
  if (b.aslda) return refresh_aslda<R>(c, b, islot, init_lam);
  if (b.cur) {
    // j of the states in the slot (Eq. jab3D; A != 1): per-state contributions
    // from the gradient launch, summed over states (before the density
    // partials, which reuse the partial-sum buffer)
    if (b.n > 0) {
      StageArgs<R> a = base_args<R>(b, box_dV(b));
      a.phi = static_cast<cx<R>*>(b.ptr(islot));
      a.h0 = static_cast<cx<R>*>(b.cur_buf);
      a.sc_in = b.sc[islot];
      a.wm = b.wm;
      a.wp = b.wp;
      wslda_status st = launch_mode<R>(c, b, MODE_GRAD, a, PROF_DENS);
      if (st) return st;
      ProfScope pj(c, PROF_DENS);
      c->launches += 2;
      CUDA_TRY(c, launch_sum_tauj<R>(static_cast<const cx<R>*>(b.cur_buf), b.n, b.M, b.nchunk, b.chunk, b.part,
                                     b.tauj, b.tauj + b.M, c->cur));
    } else {
      CUDA_TRY(c, cudaMemsetAsync(b.tauj, 0, size_t(4) * b.M * 8, c->cur));
    }
  }
  if (b.n > 0) {
    ProfScope ps(c, PROF_DENS);
    c->launches += 1;
    CUDA_TRY(c, launch_density_partial<R>(static_cast<const cx<R>*>(b.ptr(islot)), b.sc[islot],
                                          static_cast<const R*>(b.wm_r),
                                          static_cast<const R*>(b.wp_r), b.n, b.M, b.nchunk, b.chunk, b.part,
                                          c->cur));
  } else {
    CUDA_TRY(c, cudaMemsetAsync(b.part, 0, size_t(3) * b.M * b.nchunk * sizeof(double), c->cur));
  }
  {
    ProfScope ps2(c, PROF_POT);
    c->launches += 1;
    CUDA_TRY(c, launch_potentials<R>(b.part, b.nchunk, b.M, b.fdev, b.vext, b.dext, b.lam, init_lam,
                                     b.cur ? b.tauj + b.M : nullptr, b.rho, b.nu, b.U, b.delta,
                                     static_cast<fx4<R>*>(b.WD), c->cur));
    if (b.cur) {
      c->launches += 1;
      CUDA_TRY(c, launch_current_fields<R>(b.lat.nx, b.lat.ny, b.lat.nz, b.fdev.A, b.fdev.rho_floor, b.rho,
                                           b.tauj + b.M, b.d1, static_cast<fx4<R>*>(b.av), c->cur));
    }
  }
  if (b.fric && b.n > 0) {
    // per-state friction contributions (one transform pass), summed over
    // states, then added to the H fields
    StageArgs<R> a = base_args<R>(b, box_dV(b));
    a.phi = static_cast<cx<R>*>(b.ptr(islot));
    a.h0 = static_cast<cx<R>*>(b.f_scratch);
    a.sc_in = b.sc[islot];
    a.wm = b.wm;
    a.wp = b.wp;
    wslda_status st = launch_mode<R>(c, b, MODE_LAP, a, PROF_POT);
    if (st) return st;
    ProfScope ps3(c, PROF_POT);
    c->launches += 3;
    CUDA_TRY(c, launch_sum_tauj<R>(static_cast<const cx<R>*>(b.f_scratch), b.n, b.M, b.nchunk, b.chunk, b.part,
                                   b.f_div, b.f_bp, c->cur));
    CUDA_TRY(c, launch_apply_friction<R>(b.M, box_dV(b), b.f_alpha, b.f_beta, b.f_gamma, b.f_rho0, b.f_nreq, b.rho,
                                         b.nu, b.delta, b.f_div, b.f_bp, static_cast<fx4<R>*>(b.WD), c->cur));
  }
  return WSLDA_OK;
}

wslda_status refresh_fields(wslda_ctx* c, Box& b, int islot, int init_lam) {
  return c->prec == WSLDA_MIXED ? refresh_fields_t<float>(c, b, islot, init_lam)
                                : refresh_fields_t<double>(c, b, islot, init_lam);
}

template <typename R>
wslda_status stage_x(wslda_ctx* c, Box& b, double dt) {
  StageArgs<R> a = base_args<R>(b, box_dV(b));
  a.phi = static_cast<cx<R>*>(b.ptr(b.iphi));
  a.h0 = static_cast<cx<R>*>(b.ptr(b.ih[0]));
  a.h1 = static_cast<const cx<R>*>(b.ptr(b.ih[1]));
  a.h2 = static_cast<const cx<R>*>(b.ptr(b.ih[2]));
  if (b.D >= 3) a.h3 = static_cast<cx<R>*>(b.ptr(b.ih[3]));
  if (b.D >= 4) a.h4 = static_cast<cx<R>*>(b.ptr(b.ih[4]));
  a.sc_in = b.sc[b.iphi];
  a.sc_out = b.sc[b.iphi];
  a.dt = dt;
  return launch_mode<R>(c, b, x_mode(b), a, PROF_X);
}

template <typename R>
wslda_status stage_y(wslda_ctx* c, Box& b, double dt) {
  StageArgs<R> a = base_args<R>(b, box_dV(b));
  a.phi = static_cast<cx<R>*>(b.ptr(b.iphi));
  a.h3 = static_cast<cx<R>*>(b.ptr(b.ih[b.D]));  // the corrector partial
  a.sc_in = b.sc[b.iphi];
  a.sc_out = b.sc[b.iphi];
  a.dt = dt;
  return launch_mode<R>(c, b, MODE_Y, a, PROF_Y);
}

template <typename R>
wslda_status eval_f_into(wslda_ctx* c, Box& b, int in_slot, int out_slot) {
  StageArgs<R> a = base_args<R>(b, box_dV(b));
  a.phi = static_cast<cx<R>*>(b.ptr(in_slot));
  a.h0 = static_cast<cx<R>*>(b.ptr(out_slot));
  a.sc_in = b.sc[in_slot];
  a.sc_out = b.sc[out_slot];  // f is stored unscaled
  return launch_mode<R>(c, b, MODE_F, a, PROF_AUX);
}

// One Horner step out = base + coef (H - E) in (Taylor series, Eq. Taylor-exp).
template <typename R>
wslda_status horner(wslda_ctx* c, Box& b, int in_slot, int base_slot, int out_slot, double coef_im, int compute_e,
                    int normalize) {
  StageArgs<R> a = base_args<R>(b, box_dV(b));
  a.phi = static_cast<cx<R>*>(b.ptr(in_slot));
  a.h1 = static_cast<const cx<R>*>(b.ptr(base_slot));
  a.h0 = static_cast<cx<R>*>(b.ptr(out_slot));
  a.sc_in = b.sc[in_slot];
  a.sc_base = b.sc[base_slot];
  a.sc_out = b.sc[out_slot];
  a.coef_re = 0.0;
  a.coef_im = coef_im;
  a.compute_e = compute_e;
  a.normalize = normalize;
  return launch_mode<R>(c, b, MODE_HORNER, a, PROF_AUX);
}

// sum_{k=0}^{r} (-i h)^k/k! (H - E)^k phi by Horner's rule: p = phi;
// p = phi + (-i h / k) (H - E) p for k = r..1; E = <phi|H|phi> taken in the
// first application (reading T1). The result is normalised (reading T2).
template <typename R>
wslda_status taylor_series(wslda_ctx* c, Box& b, int phi_slot, int out_slot, double h, int r) {
  for (int k = r; k >= 1; --k) {
    const int in = (k == r) ? phi_slot : out_slot;
    wslda_status st = horner<R>(c, b, in, phi_slot, out_slot, -h / k, k == r, k == 1);
    if (st) return st;
  }
  return WSLDA_OK;
}

// Predictor-corrector Taylor step of Sec. 3.3 (order r = 5).
template <typename R>
wslda_status taylor_step(wslda_ctx* c, Box& b, double dt) {
  const int y = b.ih[0];
  wslda_status st;
  if ((st = taylor_series<R>(c, b, b.iphi, y, 0.5 * dt, 5))) return st;  // midpoint state
  if ((st = refresh_fields(c, b, y, 0))) return st;                      // H(t + dt/2)
  if ((st = taylor_series<R>(c, b, b.iphi, y, dt, 5))) return st;       // phi(t + dt)
  std::swap(b.iphi, b.ih[0]);
  return refresh_fields(c, b, b.iphi, 0);
}

// Autotuner: time the predictor and the corrector stage of every compiled
// launch variant of the box's shape, in both launch forms, on (a copy of) up
// to 2048 of the box's states in the free history slots, and keep the fastest
// for each stage (for boxes with current terms, each stage together with the
// current-term pass it needs and, for the predictor, the derivative launches
// of the field refreshes, which run on its variant). The choice is cached per shape, precision and state count
// for the process.
template <typename R>
wslda_status autotune_box(wslda_ctx* c, Box& b, double dt) {
  // cache: (precision, shape, states) -> (variant, persistent clusters)
  // (variant, clusters) for the predictor stage, then for the corrector stage
  static std::vector<std::pair<std::vector<int64_t>, std::vector<int>>> cache;
  if (b.n == 0) return WSLDA_OK;
  // WSLDA_VARIANT=<i> fixes the variant, WSLDA_PERSIST=0/1 the launch form
  const char* forced = getenv("WSLDA_VARIANT");
  const char* pers = getenv("WSLDA_PERSIST");
  // boxes with the current terms run their H stages one cluster per state
  const int pmode = b.cur ? 0 : (pers ? (atoi(pers) ? 1 : 0) : -1);
  std::vector<const KernelSet*> v;
  // only variants whose pencils split over the same lanes as the box's kinetic
  // tables (the frequency order of a transformed pencil depends on it)
  for (const KernelSet* k : find_variants(c->prec == WSLDA_MIXED, b.lat.nx, b.lat.ny, b.lat.nz))
    if (same_layout(k, b)) v.push_back(k);
  if (forced) v.assign(1, b.ks);
  if (v.size() == 1 && pmode >= 0) {
    b.ncl = pmode ? resident_clusters(b.ks) : 0;
    b.ks_y = b.ks;
    // WSLDA_VARIANT_Y=<j> puts the corrector stage on another variant (as the
    // autotuner may), so that mixed-variant steps can be checked
    if (const char* fy = getenv("WSLDA_VARIANT_Y")) {
      const std::vector<const KernelSet*> all =
          find_variants(c->prec == WSLDA_MIXED, b.lat.nx, b.lat.ny, b.lat.nz);
      const int i = atoi(fy);
      if (i >= 0 && i < int(all.size()) && same_layout(all[i], b)) b.ks_y = all[i];
    }
    b.ncl_y = pmode ? resident_clusters(b.ks_y) : 0;
    return WSLDA_OK;
  }
  const std::vector<int64_t> key = {c->prec, b.lat.nx, b.lat.ny, b.lat.nz, std::min<int64_t>(b.n, 2048),
                                    forced ? 1 : 0, pmode};
  for (auto& e : cache)
    if (e.first == key) {
      b.ks = v[e.second[0]];
      b.ncl = e.second[1];
      b.ks_y = v[e.second[2]];
      b.ncl_y = e.second[3];
      return WSLDA_OK;
    }
  const int64_t nt = std::min<int64_t>(b.n, 2048);
  const size_t bytes = size_t(nt) * 2 * b.M * b.csize;
  CUDA_TRY(c, cudaMemcpyAsync(b.ptr(b.ih[0]), b.ptr(b.iphi), bytes, cudaMemcpyDeviceToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(b.sc[b.ih[0]], b.sc[b.iphi], size_t(nt) * 8, cudaMemcpyDeviceToDevice, c->stream));
  for (int i = 1; i <= 2; ++i) CUDA_TRY(c, cudaMemsetAsync(b.ptr(b.ih[i]), 0, bytes, c->stream));
  cudaEvent_t e0, e1;
  CUDA_TRY(c, cudaEventCreate(&e0));
  CUDA_TRY(c, cudaEventCreate(&e1));
  int best[2] = {0, 0}, best_ncl[2] = {0, 0};
  float best_ms[2] = {1e30f, 1e30f};
  for (size_t k = 0; k < v.size(); ++k) {
    const int res = resident_clusters(v[k]);
    if (res < 1) continue;
    for (int mode = 0; mode < 2; ++mode) {
      if (pmode >= 0 && mode != pmode) continue;
      const int ncl = mode ? res : 0;
      StageArgs<R> a = base_args<R>(b, box_dV(b));
      // scratch: phi copy in ih[0], f out in ih[1], every history read and
      // the corrector partial in ih[2] (each element read, then written, by one thread)
      a.phi = static_cast<cx<R>*>(b.ptr(b.ih[0]));
      a.h0 = static_cast<cx<R>*>(b.ptr(b.ih[1]));
      a.h1 = static_cast<const cx<R>*>(b.ptr(b.ih[2]));
      a.h2 = static_cast<const cx<R>*>(b.ptr(b.ih[2]));
      a.h3 = static_cast<cx<R>*>(b.ptr(b.ih[2]));
      a.h4 = static_cast<cx<R>*>(b.ptr(b.ih[2]));
      a.sc_in = b.sc[b.ih[0]];
      a.sc_out = b.sc[b.ih[1]];
      a.dt = dt;
      a.err = c->err_d;
      // boxes with current terms: each stage comes with its current-term pass
      // (and the alpha-phi pass of ASLDA) on the same variant, and the
      // derivative launches of the field refreshes run on the predictor's
      // variant, so those are timed with the stages they go with
      StageArgs<R> g = a;
      g.h0 = static_cast<cx<R>*>(b.cur_buf);
      g.av = static_cast<const fx4<R>*>(b.av);
      g.av2 = static_cast<const fx4<R>*>(b.av_b);
      g.alf = static_cast<const cx<R>*>(b.alf);
      g.ecur = b.ecur;
      g.wm = b.wm;
      g.wp = b.wp;
      StageArgs<R> ag = a;
      ag.cur = static_cast<const cx<R>*>(b.cur_buf);
      ag.ecur = b.ecur;
      ag.alf = static_cast<const cx<R>*>(b.alf);
      for (int stage = 0; stage < 2; ++stage) {  // predictor stage, corrector stage
        const int m = stage ? int(MODE_Y) : x_mode(b);
        float ms = 1e30f;
        for (int rep = 0; rep < 4; ++rep) {
          CUDA_TRY(c, cudaEventRecord(e0, c->stream));
          if (b.cur) {
            CUDA_TRY(c, v[k]->launch[MODE_AGRAD](&g, int(nt), 0, c->stream));
            if (b.aslda) CUDA_TRY(c, v[k]->launch[MODE_KALPHA](&g, int(nt), 0, c->stream));
            CUDA_TRY(c, v[k]->launch_gen[m](&ag, int(nt), 0, c->stream));
            if (stage == 0)
              for (int r = 0; r < (b.aslda ? 4 : 2); ++r) CUDA_TRY(c, v[k]->launch[MODE_GRAD](&g, int(nt), 0, c->stream));
          } else {
            CUDA_TRY(c, v[k]->launch[m](&a, int(nt), ncl, c->stream));
          }
          CUDA_TRY(c, cudaEventRecord(e1, c->stream));
          CUDA_TRY(c, cudaEventSynchronize(e1));
          float t = 0.f;
          cudaEventElapsedTime(&t, e0, e1);
          if (rep > 0) ms = std::min(ms, t);
        }
        if (getenv("WSLDA_TUNE_VERBOSE"))
          fprintf(stderr,
                  "[wslda autotune] %dx%dx%d prec=%d %s variant %zu (cluster=%d threads=%d lanes=%d,%d,%d) "
                  "clusters=%s: %.3f ms\n",
                  b.lat.nx, b.lat.ny, b.lat.nz, c->prec, stage ? "stage Y" : "stage X", k, v[k]->cs, v[k]->bt,
                  v[k]->tx, v[k]->ty, v[k]->tz, ncl ? std::to_string(ncl).c_str() : "per-state", ms);
        // a persistent launch has to win by 3%: it is timed on fewer states
        // than it will run on, where its register spills weigh more
        if ((ncl ? 1.03f * ms : ms) < best_ms[stage]) {
          best_ms[stage] = ncl ? 1.03f * ms : ms;
          best[stage] = int(k);
          best_ncl[stage] = ncl;
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b.ks = v[best[0]];
  b.ncl = best_ncl[0];
  b.ks_y = v[best[1]];
  b.ncl_y = best_ncl[1];
  cache.push_back({key, {best[0], best_ncl[0], best[1], best_ncl[1]}});
  return WSLDA_OK;
}

// Energy terms of the current states into h[0..6] (fields must be current).
template <typename R>
wslda_status compute_energy(wslda_ctx* c, Box& b, double* h) {
  if (b.aslda) {  // every term from the per-species densities of the last refresh
    CUDA_TRY(c, launch_aslda_energy(b.M, b.rho, b.rho_b, b.nu, b.tauj, b.tauj_b, b.lam, b.vext, b.dext, b.fdev.C,
                                    b.fdev.rho_floor, box_dV(b), b.out8, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(h, b.out8, 10 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return WSLDA_OK;
  }
  StageArgs<R> a = base_args<R>(b, box_dV(b));
  a.phi = static_cast<cx<R>*>(b.ptr(b.iphi));
  a.sc_in = b.sc[b.iphi];
  c->cur = c->stream;
  wslda_status st = launch_mode<R>(c, b, MODE_EKIN, a, PROF_AUX);
  if (st) return st;
  CUDA_TRY(c, launch_energy(b.M, b.n, b.fdev, b.rho, b.nu, b.delta, b.vext, b.dext, b.ekin2, b.wm, b.wp,
                            b.cur ? b.tauj + b.M : nullptr, box_dV(b), b.out8, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(h, b.out8, 8 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return WSLDA_OK;
}

// E_tot - mu N (Eq. E_tot), with mu_a N_a + mu_b N_b for the spin-imbalanced box
double conserved_energy(const Box& b, const double* h) {
  return b.aslda ? h[5] - b.fn.mu * h[8] - b.mu_b * h[9] : h[5] - b.fn.mu * h[6];
}

template <typename R>
wslda_status start_box(wslda_ctx* c, Box& b, int stationary, double dt) {
  wslda_status st;
  if ((st = refresh_fields(c, b, b.iphi, 1))) return st;
  {
    // reference values of the conservation diagnostics (Sec. 4.5.1)
    double h[16];
    if ((st = compute_energy<R>(c, b, h))) return st;
    b.e0 = conserved_energy(b, h);
    b.n0 = h[6];
  }
  if ((st = autotune_box<R>(c, b, dt))) return st;
  const size_t bytes = size_t(b.n) * 2 * b.M * b.csize;
  if (stationary) {
    for (int i = 1; i <= b.D; ++i) CUDA_TRY(c, cudaMemsetAsync(b.ptr(b.ih[i]), 0, bytes, c->stream));
    return WSLDA_OK;
  }
  // D Taylor steps; history f(phi_0) .. f(phi_{D-1}) into ih[D] .. ih[1]
  // (oldest in ih[D]); f(phi_D) is formed by the first predictor stage.
  if ((st = eval_f_into<R>(c, b, b.iphi, b.ih[b.D]))) return st;
  for (int s = 1; s <= b.D; ++s) {
    if ((st = taylor_step<R>(c, b, dt))) return st;
    if (s < b.D && (st = eval_f_into<R>(c, b, b.iphi, b.ih[b.D - s]))) return st;
  }
  return WSLDA_OK;
}

template <typename R>
wslda_status step_box(wslda_ctx* c, Box& b, double dt) {
  wslda_status st;
  if ((st = stage_x<R>(c, b, dt))) return st;
  if ((st = refresh_fields(c, b, b.iphi, 0))) return st;
  if ((st = stage_y<R>(c, b, dt))) return st;
  if ((st = refresh_fields(c, b, b.iphi, 0))) return st;
  // Alg. 2 steps 5-7: the slot that held c becomes the slot for the next f_{k-1}
  const int freed = b.ih[b.D];
  for (int i = b.D; i >= 1; --i) b.ih[i] = b.ih[i - 1];
  b.ih[0] = freed;
  return WSLDA_OK;
}

// One AB4AM5 step of every box. With several boxes and batched execution on,
// box i runs on forked stream i mod K so that independent boxes overlap.
template <typename R>
wslda_status step_all(wslda_ctx* c, double dt) {
  wslda_status st;
  const bool fork = c->use_graph && c->boxes.size() > 1 && !c->side.empty();
  if (!fork) {
    c->cur = c->stream;
    for (Box& b : c->boxes)
      if ((st = step_box<R>(c, b, dt))) return st;
    return WSLDA_OK;
  }
  CUDA_TRY(c, cudaEventRecord(c->fork_ev, c->stream));
  for (cudaStream_t s : c->side) CUDA_TRY(c, cudaStreamWaitEvent(s, c->fork_ev, 0));
  for (size_t i = 0; i < c->boxes.size(); ++i) {
    c->cur = c->side[i % c->side.size()];
    if ((st = step_box<R>(c, c->boxes[i], dt))) {
      c->cur = c->stream;
      return st;
    }
  }
  c->cur = c->stream;
  for (size_t k = 0; k < c->side.size(); ++k) {
    CUDA_TRY(c, cudaEventRecord(c->join_ev[k], c->side[k]));
    CUDA_TRY(c, cudaStreamWaitEvent(c->stream, c->join_ev[k], 0));
  }
  return WSLDA_OK;
}

void drop_graphs(wslda_ctx* c) {
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.second);
  c->graphs.clear();
  c->graph_kernels.clear();
}

std::vector<int> slot_phase(const wslda_ctx* c) {
  std::vector<int> key;
  for (const Box& b : c->boxes) {
    key.push_back(b.iphi);
    for (int i = 0; i <= b.D; ++i) key.push_back(b.ih[i]);
  }
  return key;
}

// Four steps captured once per slot phase and dt, replayed as one graph launch.
// Capture and replay happen on a context-owned stream (the caller's stream may
// be the legacy default stream, which cannot be captured), ordered after and
// before the caller's stream with events.
template <typename R>
wslda_status step_graph4(wslda_ctx* c, double dt) {
  if (c->graph_dt != dt) {
    drop_graphs(c);
    c->graph_dt = dt;
  }
  const std::vector<int> key = slot_phase(c);
  cudaGraphExec_t exec = nullptr;
  int64_t kernels = 0;
  for (size_t i = 0; i < c->graphs.size(); ++i)
    if (c->graphs[i].first == key) {
      exec = c->graphs[i].second;
      kernels = c->graph_kernels[i];
    }
  cudaStream_t user = c->stream;
  if (!exec) {
    CUDA_TRY(c, cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
    const int64_t l0 = c->launches;
    c->stream = c->cap;
    wslda_status st = WSLDA_OK;
    for (int k = 0; k < 4 && !st; ++k) st = step_all<R>(c, dt);
    c->stream = user;
    c->cur = user;
    kernels = c->launches - l0;  // captured, not yet executed
    c->launches = l0;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->cap, &graph);
    if (st) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (e != cudaSuccess) return fail(c, WSLDA_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(c, WSLDA_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    c->graphs.push_back({key, exec});
    c->graph_kernels.push_back(kernels);
    // capture advanced the host-side slot rotation by four steps (one period
    // for AB4AM5; other schemes cycle through several captured phases)
  }
  CUDA_TRY(c, cudaEventRecord(c->cap_in, user));
  CUDA_TRY(c, cudaStreamWaitEvent(c->cap, c->cap_in, 0));
  CUDA_TRY(c, cudaGraphLaunch(exec, c->cap));
  c->launches += kernels;
  CUDA_TRY(c, cudaEventRecord(c->cap_out, c->cap));
  CUDA_TRY(c, cudaStreamWaitEvent(user, c->cap_out, 0));
  return WSLDA_OK;
}

wslda_status check_device_error(wslda_ctx* c) {
  int h = 0;
  CUDA_TRY(c, cudaMemcpyAsync(&h, c->err_d, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (h & 1) return fail(c, WSLDA_ENAN, "a state norm became non-finite or zero");
  if (h & 2) return fail(c, WSLDA_ENAN, "non-finite value in the loaded states");
  if (h & 4) return fail(c, WSLDA_ETIMEOUT, "a stage kernel's bounded wait for its slab copies gave up");
  return WSLDA_OK;
}

Box* get_box(wslda_ctx* c, int box) {
  if (box < 0 || box >= int(c->boxes.size())) return nullptr;
  return &c->boxes[box];
}

wslda_status copy_in(wslda_ctx* c, void* dst, const void* src, size_t bytes, int on_device) {
  CUDA_TRY(c, cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                              c->stream));
  return WSLDA_OK;
}

constexpr size_t kStageBytes = size_t(256) << 20;  // staging buffer for state transfers

}  // namespace

extern "C" {

int wslda_lattice_variants(int precision, int nx, int ny, int nz) {
  if (precision != WSLDA_FP64 && precision != WSLDA_MIXED) return 0;
  return int(find_variants(precision == WSLDA_MIXED, nx, ny, nz).size());
}

int wslda_lattice_supported(int precision, int nx, int ny, int nz) {
  return find_kernels(precision == WSLDA_MIXED ? 1 : 0, nx, ny, nz) != nullptr;
}

wslda_status wslda_create(int precision, void* stream, wslda_ctx** out) {
  if (!out || (precision != WSLDA_FP64 && precision != WSLDA_MIXED)) return WSLDA_EINVAL;
  wslda_ctx* c = new wslda_ctx();
  c->prec = precision;
  c->stream = static_cast<cudaStream_t>(stream);
  c->cur = c->stream;
  void* p = nullptr;
  cudaError_t e = dalloc(c, &p, sizeof(int));
  if (e != cudaSuccess) {
    delete c;
    *out = nullptr;
    return WSLDA_ECUDA;
  }
  c->err_d = static_cast<int*>(p);
  cudaMemsetAsync(c->err_d, 0, sizeof(int), c->stream);
  *out = c;
  return WSLDA_OK;
}

void wslda_destroy(wslda_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  for (void* p : c->allocs) cudaFree(p);
  for (auto& p : c->pending) {
    cudaEventDestroy(p.second.first);
    cudaEventDestroy(p.second.second);
  }
  for (cudaEvent_t e : c->evpool) cudaEventDestroy(e);
  drop_graphs(c);
  for (cudaStream_t s : c->side) cudaStreamDestroy(s);
  for (cudaEvent_t e : c->join_ev) cudaEventDestroy(e);
  if (c->fork_ev) cudaEventDestroy(c->fork_ev);
  if (c->cap) cudaStreamDestroy(c->cap);
  if (c->cap_in) cudaEventDestroy(c->cap_in);
  if (c->cap_out) cudaEventDestroy(c->cap_out);
  delete c;
}

const char* wslda_last_error(const wslda_ctx* c) {
  if (!c) return "null context";
  return c->err.empty() ? "" : c->err.c_str();
}

wslda_status wslda_set_friction(wslda_ctx* c, int box, double alpha, double beta, double gamma, double rho0,
                                double n_req) {
  CHECK_CTX(c);
  Box* b = get_box(c, box);
  if (!b) return fail(c, WSLDA_EINVAL, "set_friction: bad box");
  if (b->cur) return fail(c, WSLDA_EUNSUPPORTED, "set_friction: functional with A != 1 (or ASLDA) not supported");
  if (!std::isfinite(alpha) || !std::isfinite(beta) || !std::isfinite(gamma) || !(rho0 > 0.0) ||
      !(n_req > 0.0) || !std::isfinite(rho0) || !std::isfinite(n_req))
    return fail(c, WSLDA_EINVAL, "set_friction: coefficients must be finite, rho0 and n_req > 0");
  if (!b->f_scratch && b->n > 0) {
    const size_t sb = size_t(b->n) * 2 * b->M * b->csize;
    size_t freeb = 0, totalb = 0;
    CUDA_TRY(c, cudaMemGetInfo(&freeb, &totalb));
    if (sb + size_t(b->M) * 32 + (size_t(64) << 20) > freeb)
      return fail(c, WSLDA_ENOMEM, "set_friction: no room for the scratch state buffer");
    void* p = nullptr;
    CUDA_TRY(c, cudaMalloc(&p, sb));
    c->allocs.push_back(p);
    b->f_scratch = p;
    CUDA_TRY(c, cudaMalloc(&p, size_t(b->M) * 8));
    c->allocs.push_back(p);
    b->f_div = static_cast<double*>(p);
    CUDA_TRY(c, cudaMalloc(&p, size_t(b->M) * 24));
    c->allocs.push_back(p);
    b->f_bp = static_cast<double*>(p);
  }
  b->fric = alpha != 0.0 || beta != 0.0 || gamma != 0.0;
  b->f_alpha = alpha;
  b->f_beta = beta;
  b->f_gamma = gamma;
  b->f_rho0 = rho0;
  b->f_nreq = n_req;
  drop_graphs(c);  // captured steps hold the old field pipeline
  if (c->started && b->loaded) return refresh_fields(c, *b, b->iphi, 0);
  return WSLDA_OK;
}

wslda_status wslda_set_integrator(wslda_ctx* c, int scheme) {
  CHECK_CTX(c);
  if (!c->boxes.empty()) return fail(c, WSLDA_ESTATE, "set_integrator after add_box");
  if (scheme == WSLDA_AB4AM5) c->scheme_depth = 3;
  else if (scheme == WSLDA_AB3AM4) c->scheme_depth = 2;
  else if (scheme == WSLDA_AB5AM5) c->scheme_depth = 4;
  else return fail(c, WSLDA_EINVAL, "set_integrator: unknown scheme");
  return WSLDA_OK;
}

int wslda_add_box(wslda_ctx* c, const wslda_lattice* lat, const wslda_functional* fn, int64_t nstates) {
  if (!c) return -WSLDA_EINVAL;
  if (c->status != WSLDA_OK) return -WSLDA_ESTATE;
  if (!lat || !fn || nstates < 0) return -fail(c, WSLDA_EINVAL, "add_box: null argument or negative state count");
  if (c->started) return -fail(c, WSLDA_ESTATE, "add_box after wslda_start");
  if (lat->nx <= 0 || lat->ny <= 0 || lat->nz <= 0 || (lat->nx | lat->ny | lat->nz) & 1)
    return -fail(c, WSLDA_EINVAL, "lattice sizes must be positive and even");
  if (!(lat->dx > 0 && lat->dy > 0 && lat->dz > 0)) return -fail(c, WSLDA_EINVAL, "lattice spacings must be > 0");
  if (fn->kind != WSLDA_FUNC_SLDA_A1 && fn->kind != WSLDA_FUNC_BDG && fn->kind != WSLDA_FUNC_SLDA &&
      fn->kind != WSLDA_FUNC_ASLDA)
    return -fail(c, WSLDA_EINVAL, "unknown functional kind");
  if (fn->kind == WSLDA_FUNC_ASLDA && (!std::isfinite(fn->mu) || !std::isfinite(fn->mu_b)))
    return -fail(c, WSLDA_EINVAL, "ASLDA needs finite mu (species a) and mu_b");
  if (fn->kind != WSLDA_FUNC_BDG && !(fn->C != 0.0)) return -fail(c, WSLDA_EINVAL, "SLDA needs C != 0");
  if (fn->kind == WSLDA_FUNC_SLDA && !(fn->A > 0.0 && std::isfinite(fn->A)))
    return -fail(c, WSLDA_EINVAL, "SLDA needs a finite A > 0");
  const int prec = c->prec == WSLDA_MIXED ? 1 : 0;
  const KernelSet* ks = find_kernels(prec, lat->nx, lat->ny, lat->nz);
  if (!ks) return -fail(c, WSLDA_EUNSUPPORTED, "no compiled kernels for this lattice shape and precision");
  const int64_t M = int64_t(lat->nx) * lat->ny * lat->nz;
  if (nstates > (int64_t(1) << 31) / ks->cs - 1) return -fail(c, WSLDA_EINVAL, "too many states for one launch");

  Box b;
  b.lat = *lat;
  b.fn = *fn;
  b.n = nstates;
  b.M = int(M);
  b.ks = ks;
  b.kt[0] = ks->tx;
  b.kt[1] = ks->ty;
  b.kt[2] = ks->tz;
  b.csize = prec ? 8 : 16;
  const size_t rsize = prec ? 4 : 8;
  b.fdev.kind = fn->kind == WSLDA_FUNC_BDG ? 1 : 0;
  b.fdev.A = fn->kind == WSLDA_FUNC_SLDA ? fn->A : 1.0;  // ASLDA: unit symbol, alpha applied per site
  b.aslda = fn->kind == WSLDA_FUNC_ASLDA;
  b.mu_b = b.aslda ? fn->mu_b : fn->mu;
  b.cur = (fn->kind == WSLDA_FUNC_SLDA && fn->A != 1.0) || b.aslda;
  b.fdev.B = fn->B;
  b.fdev.C = fn->C;
  b.fdev.inv_4pi_a = fn->inv_4pi_a;
  b.fdev.mu = fn->mu;
  b.fdev.ec = fn->ec > 0 ? fn->ec : default_cutoff(*lat);
  b.fdev.rho_floor = fn->rho_floor > 0 ? fn->rho_floor : 1e-12;
  b.nchunk = density_chunks(int(M), nstates, prec == WSLDA_MIXED);
  b.chunk = std::max<int64_t>(1, (nstates + b.nchunk - 1) / b.nchunk);

  const size_t state_bytes = size_t(nstates) * 2 * M * b.csize;
  const size_t field_bytes = size_t(M) * (8 * 13 + rsize * 4) + size_t(4) * M * 8 * b.nchunk +
                             size_t(nstates) * (8 * 26 + rsize * 2) + 4096;
  const int D = c->scheme_depth;
  const size_t need = size_t(D + 2 + (b.cur ? 1 : 0)) * state_bytes + field_bytes +
                      (b.cur ? size_t(M) * (32 + 4 * rsize) + size_t(nstates) * 128 : 0) +
                      (b.aslda ? size_t(M) * (8 * 14 + rsize * 6) + size_t(4) * M * 8 * b.nchunk +
                                     size_t(nstates) * (8 + rsize) : 0);
  size_t freeb = 0, totalb = 0;
  CUDA_TRY_NEG(c, cudaMemGetInfo(&freeb, &totalb));
  const size_t margin = size_t(1) << 30;
  if (need + margin > freeb) {
    fail(c, WSLDA_ENOMEM, "box needs " + std::to_string(need >> 20) + " MiB, " + std::to_string(freeb >> 20) +
                              " MiB free");
    return -WSLDA_ENOMEM;
  }
  if (resident_clusters(ks) < 1)
    return -fail(c, WSLDA_EUNSUPPORTED, "stage kernel cannot be resident on this device");

#define ALLOC(ptr, bytes)                                                            \
  do {                                                                               \
    void* p_ = nullptr;                                                              \
    cudaError_t e_ = dalloc(c, &p_, (bytes));                                        \
    if (e_ != cudaSuccess) {                                                         \
      fail(c, WSLDA_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e_));  \
      return -WSLDA_ENOMEM;                                                          \
    }                                                                                \
    ptr = decltype(ptr)(p_);                                                         \
  } while (0)

  b.D = D;
  for (int i = 0; i < D + 2; ++i) ALLOC(b.slot[i], state_bytes);
  ALLOC(b.vext, M * 8);
  ALLOC(b.dext, 2 * M * 8);
  ALLOC(b.lam, M * 8);
  ALLOC(b.rho, M * 8);
  ALLOC(b.nu, 2 * M * 8);
  ALLOC(b.U, M * 8);
  ALLOC(b.delta, 2 * M * 8);
  ALLOC(b.WD, 4 * M * rsize);
  for (int i = 0; i < D + 2; ++i) ALLOC(b.sc[i], std::max<int64_t>(nstates, 1) * 8);
  const int naxis = lat->nx + lat->ny + lat->nz;
  ALLOC(b.ktab, 2 * naxis * rsize);
  ALLOC(b.tw, 2 * naxis * rsize);
  ALLOC(b.wm, std::max<int64_t>(nstates, 1) * 8);
  ALLOC(b.wp, std::max<int64_t>(nstates, 1) * 8);
  ALLOC(b.wm_r, std::max<int64_t>(nstates, 1) * rsize);
  ALLOC(b.wp_r, std::max<int64_t>(nstates, 1) * rsize);
  ALLOC(b.part, size_t(4) * M * 8 * b.nchunk);
  ALLOC(b.Ebuf, std::max<int64_t>(nstates, 1) * 8);
  ALLOC(b.npart, std::max<int64_t>(nstates, 1) * 16 * 8);
  ALLOC(b.ekin2, std::max<int64_t>(nstates, 1) * 16);
  ALLOC(b.out8, 16 * 8);
  if (b.cur) {
    ALLOC(b.cur_buf, std::max<size_t>(state_bytes, 16));
    ALLOC(b.tauj, size_t(4) * M * 8);
    ALLOC(b.av, size_t(4) * M * rsize);
    ALLOC(b.ecur, std::max<int64_t>(nstates, 1) * 16 * 8);
    ALLOC(b.d1, size_t(lat->nx + lat->ny + lat->nz) * 8);
  }
  if (b.aslda) {
    ALLOC(b.tauj_b, size_t(4) * M * 8);
    ALLOC(b.rho_b, M * 8);
    ALLOC(b.U_b, M * 8);
    ALLOC(b.d2, size_t(lat->nx + lat->ny + lat->nz) * 8);
    ALLOC(b.af, size_t(8) * M * 8);
    ALLOC(b.part_b, size_t(4) * M * 8 * b.nchunk);
    ALLOC(b.av_b, size_t(4) * M * rsize);
    ALLOC(b.alf, size_t(2) * M * rsize);
    ALLOC(b.wzero, std::max<int64_t>(nstates, 1) * 8);
    ALLOC(b.wzero_r, std::max<int64_t>(nstates, 1) * rsize);
    CUDA_TRY_NEG(c, cudaMemsetAsync(b.wzero, 0, std::max<int64_t>(nstates, 1) * 8, c->stream));
    CUDA_TRY_NEG(c, cudaMemsetAsync(b.wzero_r, 0, std::max<int64_t>(nstates, 1) * rsize, c->stream));
  }
#undef ALLOC
  CUDA_TRY_NEG(c, cudaMemsetAsync(b.vext, 0, M * 8, c->stream));
  CUDA_TRY_NEG(c, cudaMemsetAsync(b.dext, 0, 2 * M * 8, c->stream));

  // kinetic symbol k_d^2 * 0.5 / M per slot (1/M folds in the unnormalised inverse FFT)
  std::vector<double> k2, k1, twr, twi;
  const double scale = 0.5 / double(M);
  axis_tables(lat->nx, ks->tx, lat->dx, scale, k2, k1, twr, twi);
  axis_tables(lat->ny, ks->ty, lat->dy, scale, k2, k1, twr, twi);
  axis_tables(lat->nz, ks->tz, lat->dz, scale, k2, k1, twr, twi);
  // constant inverse effective mass: -1/2 grad.alpha grad = -alpha/2 lap (Eq. kinop-alpha)
  for (double& v : k2) v *= b.fdev.A;
  k2.insert(k2.end(), k1.begin(), k1.end());
  if (b.cur) {
    // first column of the periodic first-derivative matrix of each axis with
    // the Nyquist mode left out: d_j = -(2/N) sum_{m=1}^{N/2-1} k_m sin(2 pi m j / N)
    std::vector<double> d1;
    const int ns[3] = {lat->nx, lat->ny, lat->nz};
    const double ds[3] = {lat->dx, lat->dy, lat->dz};
    for (int ax = 0; ax < 3; ++ax) {
      const int N = ns[ax];
      for (int jj = 0; jj < N; ++jj) {
        double acc = 0.0;
        for (int m = 1; m < N / 2; ++m)
          acc -= 2.0 * (2.0 * M_PI * m / (N * ds[ax])) * sin(2.0 * M_PI * double(m) * double(jj) / double(N));
        d1.push_back(acc / N);
      }
    }
    CUDA_TRY_NEG(c, cudaMemcpyAsync(b.d1, d1.data(), d1.size() * 8, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY_NEG(c, cudaStreamSynchronize(c->stream));
  }
  if (b.aslda) {
    // first column of the periodic second-derivative matrix of Eq. D2 (the
    // Laplacian of H, Nyquist mode kept): c_j = -(1/N) sum_m k_m^2 cos(2 pi m j / N)
    std::vector<double> d2;
    const int ns[3] = {lat->nx, lat->ny, lat->nz};
    const double ds[3] = {lat->dx, lat->dy, lat->dz};
    for (int ax = 0; ax < 3; ++ax) {
      const int N = ns[ax];
      for (int jj = 0; jj < N; ++jj) {
        double acc = 0.0;
        for (int m = 0; m < N; ++m) {
          const int f = m <= N / 2 ? m : m - N;
          const double k = 2.0 * M_PI * f / (N * ds[ax]);
          acc -= k * k * cos(2.0 * M_PI * double((int64_t(m) * jj) % N) / double(N));
        }
        d2.push_back(acc / N);
      }
    }
    CUDA_TRY_NEG(c, cudaMemcpyAsync(b.d2, d2.data(), d2.size() * 8, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY_NEG(c, cudaStreamSynchronize(c->stream));
  }
  std::vector<double> tw(2 * naxis);
  for (int i = 0; i < naxis; ++i) {
    tw[2 * i] = twr[i];
    tw[2 * i + 1] = twi[i];
  }
  void* tmp = nullptr;
  CUDA_TRY_NEG(c, cudaMalloc(&tmp, 4 * naxis * 8));
  cudaMemcpyAsync(tmp, k2.data(), 2 * naxis * 8, cudaMemcpyHostToDevice, c->stream);
  cudaMemcpyAsync(static_cast<char*>(tmp) + 2 * naxis * 8, tw.data(), 2 * naxis * 8, cudaMemcpyHostToDevice,
                  c->stream);
  if (prec) {
    launch_to_real<float>(static_cast<double*>(tmp), static_cast<float*>(b.ktab), 2 * naxis, c->stream);
    launch_to_real<float>(static_cast<double*>(tmp) + 2 * naxis, static_cast<float*>(b.tw), 2 * naxis, c->stream);
  } else {
    cudaMemcpyAsync(b.ktab, tmp, 2 * naxis * 8, cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(b.tw, static_cast<double*>(tmp) + 2 * naxis, 2 * naxis * 8, cudaMemcpyDeviceToDevice,
                    c->stream);
  }
  CUDA_TRY_NEG(c, cudaStreamSynchronize(c->stream));
  cudaFree(tmp);
  c->boxes.push_back(b);
  return int(c->boxes.size()) - 1;
}

wslda_status wslda_set_vext(wslda_ctx* c, int box, const double* vext, int on_device) {
  CHECK_CTX(c);
  Box* b = get_box(c, box);
  if (!b || !vext) return fail(c, WSLDA_EINVAL, "set_vext: bad box or null pointer");
  if (c->started) return fail(c, WSLDA_ESTATE, "set_vext after wslda_start");
  return copy_in(c, b->vext, vext, size_t(b->M) * 8, on_device);
}

wslda_status wslda_set_dext(wslda_ctx* c, int box, const double* dext, int on_device) {
  CHECK_CTX(c);
  Box* b = get_box(c, box);
  if (!b || !dext) return fail(c, WSLDA_EINVAL, "set_dext: bad box or null pointer");
  if (c->started) return fail(c, WSLDA_ESTATE, "set_dext after wslda_start");
  return copy_in(c, b->dext, dext, size_t(b->M) * 16, on_device);
}

// Frozen weights (T = 0 when NULL) in double and in the working precision;
// then the device error word (non-finite loaded states) is checked.
static wslda_status set_weights(wslda_ctx* c, Box& bx, const double* w_minus, const double* w_plus) {
  Box* b = &bx;
  std::vector<double> wm(std::max<int64_t>(b->n, 1), 1.0), wp(std::max<int64_t>(b->n, 1), 0.0);
  for (int64_t i = 0; i < b->n; ++i) {
    if (w_minus) wm[i] = w_minus[i];
    if (w_plus) wp[i] = w_plus[i];
    if (!std::isfinite(wm[i]) || !std::isfinite(wp[i])) return fail(c, WSLDA_ENAN, "non-finite weight");
  }
  CUDA_TRY(c, cudaMemcpyAsync(b->wm, wm.data(), wm.size() * 8, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(b->wp, wp.data(), wp.size() * 8, cudaMemcpyHostToDevice, c->stream));
  if (c->prec == WSLDA_MIXED) {
    CUDA_TRY(c, launch_to_real<float>(b->wm, static_cast<float*>(b->wm_r), int64_t(wm.size()), c->stream));
    CUDA_TRY(c, launch_to_real<float>(b->wp, static_cast<float*>(b->wp_r), int64_t(wp.size()), c->stream));
  } else {
    CUDA_TRY(c, cudaMemcpyAsync(b->wm_r, b->wm, wm.size() * 8, cudaMemcpyDeviceToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(b->wp_r, b->wp, wp.size() * 8, cudaMemcpyDeviceToDevice, c->stream));
  }
  wslda_status st = check_device_error(c);
  if (st) return st;
  b->loaded = true;
  return WSLDA_OK;
}

wslda_status wslda_load_states(wslda_ctx* c, int box, const double* uv, const double* w_minus, const double* w_plus,
                               int on_device) {
  CHECK_CTX(c);
  Box* b = get_box(c, box);
  if (!b || (!uv && b->n > 0)) return fail(c, WSLDA_EINVAL, "load_states: bad box or null pointer");
  if (c->started) return fail(c, WSLDA_ESTATE, "load_states after wslda_start");
  const int64_t total = b->n * 2 * int64_t(b->M);  // complex elements
  const int64_t per = int64_t(kStageBytes / 16);
  void* stage = nullptr;
  if (total > 0) CUDA_TRY(c, cudaMalloc(&stage, size_t(std::min(total, per)) * 16));
  for (int64_t off = 0; off < total; off += per) {
    const int64_t cnt = std::min(per, total - off);
    const double* src = uv + 2 * off;
    const double* dsrc = src;
    if (!on_device) {
      CUDA_TRY(c, cudaMemcpyAsync(stage, src, cnt * 16, cudaMemcpyHostToDevice, c->stream));
      dsrc = static_cast<const double*>(stage);
    }
    cudaError_t e;
    if (c->prec == WSLDA_MIXED)
      e = launch_narrow<float>(dsrc, static_cast<float2*>(b->slot[b->iphi]) + off, cnt, c->err_d, c->stream);
    else
      e = launch_narrow<double>(dsrc, static_cast<double2*>(b->slot[b->iphi]) + off, cnt, c->err_d, c->stream);
    if (e != cudaSuccess) {
      cudaFree(stage);
      return fail(c, WSLDA_ECUDA, std::string("narrow: ") + cudaGetErrorString(e));
    }
  }
  CUDA_TRY(c, launch_fill(b->sc[b->iphi], 1.0, std::max<int64_t>(b->n, 1), c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (stage) cudaFree(stage);
  return set_weights(c, *b, w_minus, w_plus);
}

wslda_status wslda_fill_uniform_states(wslda_ctx* c, int box, double mu_eff, double delta, const int64_t* kidx) {
  CHECK_CTX(c);
  Box* b = get_box(c, box);
  if (!b) return fail(c, WSLDA_EINVAL, "fill_uniform_states: bad box");
  if (c->started) return fail(c, WSLDA_ESTATE, "fill_uniform_states after wslda_start");
  if (!(delta > 0.0) || !std::isfinite(mu_eff)) return fail(c, WSLDA_EINVAL, "fill_uniform_states: need delta > 0");
  // an ASLDA box takes n/2 positive-energy states and their partners
  const int64_t nk = b->aslda ? b->n / 2 : b->n;
  if (b->aslda && (b->n & 1)) return fail(c, WSLDA_EINVAL, "fill_uniform_states: an ASLDA box needs an even count");
  if (!kidx && nk > b->M) return fail(c, WSLDA_EINVAL, "more states than lattice momenta");
  int64_t* kd = nullptr;
  if (kidx && nk > 0) {
    for (int64_t i = 0; i < nk; ++i)
      if (kidx[i] < 0 || kidx[i] >= b->M) return fail(c, WSLDA_EINVAL, "k index out of range");
    CUDA_TRY(c, cudaMalloc(&kd, size_t(nk) * 8));
    CUDA_TRY(c, cudaMemcpyAsync(kd, kidx, size_t(nk) * 8, cudaMemcpyHostToDevice, c->stream));
  }
  cudaError_t e = launch_fill_plane_waves(b->slot[b->iphi], c->prec == WSLDA_MIXED, b->lat, mu_eff, delta, kd, b->n,
                                          b->aslda ? 1 : 0, c->stream);
  if (e == cudaSuccess) e = launch_fill(b->sc[b->iphi], 1.0, std::max<int64_t>(b->n, 1), c->stream);
  cudaError_t e2 = cudaStreamSynchronize(c->stream);
  if (kd) cudaFree(kd);
  if (e != cudaSuccess || e2 != cudaSuccess)
    return fail(c, WSLDA_ECUDA, std::string("fill_uniform_states: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
  std::vector<double> wm(std::max<int64_t>(b->n, 1), 1.0), wp(std::max<int64_t>(b->n, 1), 0.0);
  for (int64_t i = nk; i < b->n; ++i) {  // T = 0: the partners (E < 0) have f(E) = 1, f(-E) = 0
    wm[i] = 0.0;
    wp[i] = 1.0;
  }
  CUDA_TRY(c, cudaMemcpyAsync(b->wm, wm.data(), wm.size() * 8, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(b->wp, wp.data(), wp.size() * 8, cudaMemcpyHostToDevice, c->stream));
  if (c->prec == WSLDA_MIXED) {
    CUDA_TRY(c, launch_to_real<float>(b->wm, static_cast<float*>(b->wm_r), int64_t(wm.size()), c->stream));
    CUDA_TRY(c, launch_to_real<float>(b->wp, static_cast<float*>(b->wp_r), int64_t(wp.size()), c->stream));
  } else {
    CUDA_TRY(c, cudaMemcpyAsync(b->wm_r, b->wm, wm.size() * 8, cudaMemcpyDeviceToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(b->wp_r, b->wp, wp.size() * 8, cudaMemcpyDeviceToDevice, c->stream));
  }
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  b->loaded = true;
  return WSLDA_OK;
}

wslda_status wslda_set_weights(wslda_ctx* c, int box, const double* w_minus, const double* w_plus) {
  CHECK_CTX(c);
  Box* b = get_box(c, box);
  if (!b) return fail(c, WSLDA_EINVAL, "set_weights: bad box");
  if (!b->loaded) return fail(c, WSLDA_ESTATE, "set_weights before the states are loaded");
  if (c->started) return fail(c, WSLDA_ESTATE, "set_weights after wslda_start");
  return set_weights(c, *b, w_minus, w_plus);
}

wslda_status wslda_imprint_phase(wslda_ctx* c, int box, int comp, const double* phase, int on_device) {
  CHECK_CTX(c);
  Box* b = get_box(c, box);
  if (!b || !phase || (comp != 0 && comp != 1)) return fail(c, WSLDA_EINVAL, "imprint_phase: bad box, component or pointer");
  if (!b->loaded) return fail(c, WSLDA_ESTATE, "imprint_phase before the states are loaded");
  if (c->started) return fail(c, WSLDA_ESTATE, "imprint_phase after wslda_start");
  const size_t bytes = size_t(b->M) * 16;
  const double* dph = phase;
  void* tmp = nullptr;
  if (!on_device) {
    for (size_t i = 0; i < 2 * size_t(b->M); ++i)
      if (!std::isfinite(phase[i])) return fail(c, WSLDA_ENAN, "imprint_phase: non-finite phase");
    CUDA_TRY(c, cudaMalloc(&tmp, bytes));
    cudaError_t e = cudaMemcpyAsync(tmp, phase, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) {
      cudaFree(tmp);
      return fail(c, WSLDA_ECUDA, std::string("imprint_phase: ") + cudaGetErrorString(e));
    }
    dph = static_cast<const double*>(tmp);
  }
  // the deferred normalisation factor multiplies the whole state, so it commutes with the phase
  cudaError_t e = c->prec == WSLDA_MIXED
                      ? launch_imprint<float>(static_cast<float2*>(b->slot[b->iphi]), b->n, b->M, comp, dph, c->stream)
                      : launch_imprint<double>(static_cast<double2*>(b->slot[b->iphi]), b->n, b->M, comp, dph,
                                               c->stream);
  cudaError_t e2 = cudaStreamSynchronize(c->stream);
  if (tmp) cudaFree(tmp);
  if (e != cudaSuccess || e2 != cudaSuccess)
    return fail(c, WSLDA_ECUDA, std::string("imprint_phase: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
  return WSLDA_OK;
}

namespace {
// max |x[i] - x[mirror(i)]| over the reflections i -> N - i (mod N) of each axis
double mirror_asymmetry(const double* x, int stride, const wslda_lattice& l) {
  double worst = 0.0;
  for (int ix = 0; ix < l.nx; ++ix)
    for (int iy = 0; iy < l.ny; ++iy)
      for (int iz = 0; iz < l.nz; ++iz) {
        const int s = (ix * l.ny + iy) * l.nz + iz;
        const int rx = (l.nx - ix) % l.nx, ry = (l.ny - iy) % l.ny, rz = (l.nz - iz) % l.nz;
        const int m[3] = {(rx * l.ny + iy) * l.nz + iz, (ix * l.ny + ry) * l.nz + iz, (ix * l.ny + iy) * l.nz + rz};
        for (int k = 0; k < 3; ++k) worst = std::max(worst, std::fabs(x[size_t(s) * stride] - x[size_t(m[k]) * stride]));
      }
  return worst;
}
double max_abs(const double* x, size_t n) {
  double m = 0.0;
  for (size_t i = 0; i < n; ++i) m = std::max(m, std::fabs(x[i]));
  return m;
}
}  // namespace

wslda_status wslda_static_solve(wslda_ctx* c, int box, const double* U0, const double* delta0,
                                const wslda_scf_params* p, double* qp_energies, wslda_scf_result* out) {
  CHECK_CTX(c);
  Box* b = get_box(c, box);
  if (!b || !U0 || !delta0 || !p || !out) return fail(c, WSLDA_EINVAL, "static_solve: bad box or null pointer");
  if (c->started) return fail(c, WSLDA_ESTATE, "static_solve after wslda_start");
  if (b->n != b->M) return fail(c, WSLDA_EINVAL, "static_solve: the box must hold nstates = M states");
  if (b->fdev.A != 1.0 || b->aslda)
    return fail(c, WSLDA_EUNSUPPORTED, "static_solve: functional with A != 1 (or ASLDA) not built");
  if (!(p->mixing > 0.0 && p->mixing <= 1.0) || p->max_iters < 1 || !(p->eps_energy >= 0.0) ||
      !std::isfinite(p->e_ref) || !std::isfinite(p->n_target) || !std::isfinite(p->a_mu) ||
      (p->n_target > 0 && !(p->eps_npart > 0.0)) || (p->method != 0 && p->method != 1) ||
      !std::isfinite(p->broyden_w0) || p->fp32_iters < 0)
    return fail(c, WSLDA_EINVAL, "static_solve: bad parameters");
  const size_t M = size_t(b->M);
  std::vector<double> v(M), d(2 * M);
  CUDA_TRY(c, cudaMemcpyAsync(v.data(), b->vext, M * 8, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(d.data(), b->dext, 2 * M * 8, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (max_abs(d.data(), d.size()) != 0.0)
    return fail(c, WSLDA_EINVAL, "static_solve: an external pairing field is not supported");
  for (size_t i = 0; i < M; ++i)
    if (!std::isfinite(U0[i]) || !std::isfinite(delta0[i])) return fail(c, WSLDA_ENAN, "static_solve: non-finite input");
  const double* arrs[3] = {v.data(), U0, delta0};
  for (const double* x : arrs)
    if (mirror_asymmetry(x, 1, b->lat) > 1e-12 * std::max(1.0, max_abs(x, M)))
      return fail(c, WSLDA_EINVAL, "static_solve: V_ext, U0 and delta0 must be symmetric about site N/2 on every axis");
  ScfBox view{b->lat, b->fdev, b->M, c->prec, b->slot[b->iphi], b->sc[b->iphi], b->vext, b->dext, b->rho, b->nu,
              b->delta, b->ekin2, b->wm, b->wp, b->out8, c->stream};
  std::string err;
  const wslda_status st = static_solve(view, U0, delta0, *p, qp_energies, out, err);
  if (st != WSLDA_OK) return fail(c, st, "static_solve: " + err);
  b->fn.mu = out->mu;
  b->fdev.mu = out->mu;
  if (c->prec == WSLDA_MIXED) {
    CUDA_TRY(c, launch_to_real<float>(b->wm, static_cast<float*>(b->wm_r), b->n, c->stream));
    CUDA_TRY(c, launch_to_real<float>(b->wp, static_cast<float*>(b->wp_r), b->n, c->stream));
  } else {
    CUDA_TRY(c, cudaMemcpyAsync(b->wm_r, b->wm, size_t(b->n) * 8, cudaMemcpyDeviceToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(b->wp_r, b->wp, size_t(b->n) * 8, cudaMemcpyDeviceToDevice, c->stream));
  }
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  b->loaded = true;
  return WSLDA_OK;
}

wslda_status wslda_start(wslda_ctx* c, int stationary, double dt) {
  CHECK_CTX(c);
  if (!(dt != 0.0) || !std::isfinite(dt)) return fail(c, WSLDA_EINVAL, "dt must be finite and non-zero");
  if (c->boxes.empty()) return fail(c, WSLDA_ESTATE, "no boxes");
  for (Box& b : c->boxes)
    if (!b.loaded) return fail(c, WSLDA_ESTATE, "wslda_start before load_states");
  wslda_status st;
  for (Box& b : c->boxes) {
    st = c->prec == WSLDA_MIXED ? start_box<float>(c, b, stationary, dt) : start_box<double>(c, b, stationary, dt);
    if (st) return st;
  }
  collect_profile(c);
  if ((st = check_device_error(c))) return st;
  drop_graphs(c);
  c->started = true;
  c->dt_start = dt;
  c->t = stationary ? 0.0 : c->scheme_depth * dt;  // one Taylor step per history value
  c->steps = stationary ? 0 : c->scheme_depth;
  return WSLDA_OK;
}

wslda_status wslda_step(wslda_ctx* c, double dt, int nsteps) {
  CHECK_CTX(c);
  if (!c->started) return fail(c, WSLDA_ESTATE, "wslda_step before wslda_start");
  if (nsteps < 0) return fail(c, WSLDA_EINVAL, "nsteps < 0");
  if (dt != c->dt_start) return fail(c, WSLDA_EINVAL, "dt differs from the start-up dt; call wslda_start again");
  int done = 0;
  if (c->use_graph && !c->prof) {
    for (; done + 4 <= nsteps; done += 4) {
      wslda_status st = c->prec == WSLDA_MIXED ? step_graph4<float>(c, dt) : step_graph4<double>(c, dt);
      if (st) return st;
    }
  }
  for (int i = done; i < nsteps; ++i) {
    wslda_status st = c->prec == WSLDA_MIXED ? step_all<float>(c, dt) : step_all<double>(c, dt);
    if (st) return st;
    if (c->prof && c->pending.size() > 4096) collect_profile(c);
  }
  collect_profile(c);
  wslda_status st = check_device_error(c);
  if (st) return st;
  c->t += nsteps * dt;
  c->steps += nsteps;
  return WSLDA_OK;
}

wslda_status wslda_get_states(wslda_ctx* c, int box, double* uv, int on_device) {
  CHECK_CTX(c);
  Box* b = get_box(c, box);
  if (!b || (!uv && b->n > 0)) return fail(c, WSLDA_EINVAL, "get_states: bad box or null pointer");
  const int64_t total = b->n * 2 * int64_t(b->M);
  const int64_t per = int64_t(kStageBytes / 16);
  void* stage = nullptr;
  if (total > 0 && !on_device) CUDA_TRY(c, cudaMalloc(&stage, size_t(std::min(total, per)) * 16));
  for (int64_t off = 0; off < total; off += per) {
    const int64_t cnt = std::min(per, total - off);
    double* dst = on_device ? uv + 2 * off : static_cast<double*>(stage);
    const int64_t per_state = 2 * int64_t(b->M);
    cudaError_t e = c->prec == WSLDA_MIXED
                        ? launch_widen<float>(static_cast<float2*>(b->slot[b->iphi]) + off, dst, cnt, b->sc[b->iphi],
                                              off, per_state, c->stream)
                        : launch_widen<double>(static_cast<double2*>(b->slot[b->iphi]) + off, dst, cnt,
                                               b->sc[b->iphi], off, per_state, c->stream);
    if (e != cudaSuccess) {
      if (stage) cudaFree(stage);
      return fail(c, WSLDA_ECUDA, std::string("widen: ") + cudaGetErrorString(e));
    }
    if (!on_device) CUDA_TRY(c, cudaMemcpyAsync(uv + 2 * off, stage, cnt * 16, cudaMemcpyDeviceToHost, c->stream));
  }
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (stage) cudaFree(stage);
  return WSLDA_OK;
}

wslda_status wslda_load_states_f32(wslda_ctx* c, int box, const float* uv, const double* w_minus,
                                   const double* w_plus, int on_device) {
  CHECK_CTX(c);
  Box* b = get_box(c, box);
  if (!b || (!uv && b->n > 0)) return fail(c, WSLDA_EINVAL, "load_states_f32: bad box or null pointer");
  if (c->started) return fail(c, WSLDA_ESTATE, "load_states_f32 after wslda_start");
  const int64_t total = b->n * 2 * int64_t(b->M);  // complex elements
  const int64_t per = int64_t(kStageBytes / 8);
  const float2* src = reinterpret_cast<const float2*>(uv);
  void* stage = nullptr;
  if (total > 0 && !on_device && c->prec != WSLDA_MIXED)
    CUDA_TRY(c, cudaMalloc(&stage, size_t(std::min(total, per)) * 8));
  for (int64_t off = 0; off < total; off += per) {
    const int64_t cnt = std::min(per, total - off);
    const float2* dsrc = src + off;
    cudaError_t e = cudaSuccess;
    if (!on_device) {
      if (c->prec == WSLDA_MIXED) {  // straight into the state slot, then checked in place
        e = cudaMemcpyAsync(static_cast<float2*>(b->slot[b->iphi]) + off, dsrc, cnt * 8, cudaMemcpyHostToDevice,
                            c->stream);
        dsrc = static_cast<const float2*>(b->slot[b->iphi]) + off;
      } else {
        e = cudaMemcpyAsync(stage, dsrc, cnt * 8, cudaMemcpyHostToDevice, c->stream);
        dsrc = static_cast<const float2*>(stage);
      }
    }
    if (e == cudaSuccess)
      e = c->prec == WSLDA_MIXED
              ? launch_rescale<float2, float2>(dsrc, static_cast<float2*>(b->slot[b->iphi]) + off, cnt, nullptr, 0,
                                               1, c->err_d, c->stream)
              : launch_rescale<float2, double2>(dsrc, static_cast<double2*>(b->slot[b->iphi]) + off, cnt, nullptr, 0,
                                                1, c->err_d, c->stream);
    if (e != cudaSuccess) {
      if (stage) cudaFree(stage);
      return fail(c, WSLDA_ECUDA, std::string("load_states_f32: ") + cudaGetErrorString(e));
    }
  }
  CUDA_TRY(c, launch_fill(b->sc[b->iphi], 1.0, std::max<int64_t>(b->n, 1), c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (stage) cudaFree(stage);
  return set_weights(c, *b, w_minus, w_plus);
}

wslda_status wslda_get_states_f32(wslda_ctx* c, int box, float* uv, int on_device) {
  CHECK_CTX(c);
  Box* b = get_box(c, box);
  if (!b || (!uv && b->n > 0)) return fail(c, WSLDA_EINVAL, "get_states_f32: bad box or null pointer");
  const int64_t total = b->n * 2 * int64_t(b->M);
  const int64_t per = int64_t(kStageBytes / 8);
  const int64_t per_state = 2 * int64_t(b->M);
  float2* out = reinterpret_cast<float2*>(uv);
  void* stage = nullptr;
  if (total > 0 && !on_device) CUDA_TRY(c, cudaMalloc(&stage, size_t(std::min(total, per)) * 8));
  for (int64_t off = 0; off < total; off += per) {
    const int64_t cnt = std::min(per, total - off);
    float2* dst = on_device ? out + off : static_cast<float2*>(stage);
    cudaError_t e = c->prec == WSLDA_MIXED
                        ? launch_rescale<float2, float2>(static_cast<const float2*>(b->slot[b->iphi]) + off, dst, cnt,
                                                         b->sc[b->iphi], off, per_state, nullptr, c->stream)
                        : launch_rescale<double2, float2>(static_cast<const double2*>(b->slot[b->iphi]) + off, dst,
                                                          cnt, b->sc[b->iphi], off, per_state, nullptr, c->stream);
    if (e == cudaSuccess && !on_device)
      e = cudaMemcpyAsync(out + off, stage, cnt * 8, cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) {
      if (stage) cudaFree(stage);
      return fail(c, WSLDA_ECUDA, std::string("get_states_f32: ") + cudaGetErrorString(e));
    }
  }
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (stage) cudaFree(stage);
  return WSLDA_OK;
}

wslda_status wslda_get_densities(wslda_ctx* c, int box, double* rho, double* nu, double* tau, double* j) {
  CHECK_CTX(c);
  Box* b = get_box(c, box);
  if (!b) return fail(c, WSLDA_EINVAL, "get_densities: bad box");
  if (!b->loaded) return fail(c, WSLDA_ESTATE, "get_densities before load_states");
  if (!c->started) {
    // densities of the loaded states (regulator from the t = 0 fixed point)
    wslda_status st = refresh_fields(c, *b, b->iphi, 1);
    if (st) return st;
  }
  if (b->aslda) {  // spin average of rho; tau and j per species come from wslda_get_spin_densities
    if (tau || j) return fail(c, WSLDA_EINVAL, "get_densities: tau / j of an ASLDA box: use get_spin_densities");
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (rho) {
      std::vector<double> ra(b->M), rb(b->M);
      CUDA_TRY(c, cudaMemcpy(ra.data(), b->rho, size_t(b->M) * 8, cudaMemcpyDeviceToHost));
      CUDA_TRY(c, cudaMemcpy(rb.data(), b->rho_b, size_t(b->M) * 8, cudaMemcpyDeviceToHost));
      for (int i = 0; i < b->M; ++i) rho[i] = 0.5 * (ra[i] + rb[i]);
    }
    if (nu) CUDA_TRY(c, cudaMemcpy(nu, b->nu, size_t(b->M) * 16, cudaMemcpyDeviceToHost));
    return WSLDA_OK;
  }
  if (rho) CUDA_TRY(c, cudaMemcpyAsync(rho, b->rho, size_t(b->M) * 8, cudaMemcpyDeviceToHost, c->stream));
  if (nu) CUDA_TRY(c, cudaMemcpyAsync(nu, b->nu, size_t(b->M) * 16, cudaMemcpyDeviceToHost, c->stream));
  if ((tau || j) && b->n > 0) {
    // the gradient launch leaves per-state contributions in the free history
    // slot (between steps slot ih[0] holds nothing live), then a site-major
    // sum over states; tau_d and j_d use the Nyquist-free gradient
    wslda_status st;
    c->cur = c->stream;
    if (c->prec == WSLDA_MIXED) {
      StageArgs<float> a = base_args<float>(*b, box_dV(*b));
      a.phi = static_cast<float2*>(b->ptr(b->iphi));
      a.h0 = static_cast<float2*>(b->ptr(b->ih[0]));
      a.sc_in = b->sc[b->iphi];
      a.wm = b->wm;
      a.wp = b->wp;
      if ((st = launch_mode<float>(c, *b, MODE_GRAD, a, PROF_AUX))) return st;
    } else {
      StageArgs<double> a = base_args<double>(*b, box_dV(*b));
      a.phi = static_cast<double2*>(b->ptr(b->iphi));
      a.h0 = static_cast<double2*>(b->ptr(b->ih[0]));
      a.sc_in = b->sc[b->iphi];
      a.wm = b->wm;
      a.wp = b->wp;
      if ((st = launch_mode<double>(c, *b, MODE_GRAD, a, PROF_AUX))) return st;
    }
    double* tj = nullptr;
    CUDA_TRY(c, cudaMalloc(&tj, size_t(4) * b->M * 8));
    cudaError_t e = c->prec == WSLDA_MIXED
                        ? launch_sum_tauj<float>(static_cast<const float2*>(b->ptr(b->ih[0])), b->n, b->M, b->nchunk,
                                                 b->chunk, b->part, tj, tj + b->M, c->stream)
                        : launch_sum_tauj<double>(static_cast<const double2*>(b->ptr(b->ih[0])), b->n, b->M,
                                                  b->nchunk, b->chunk, b->part, tj, tj + b->M, c->stream);
    if (e == cudaSuccess && tau) e = cudaMemcpyAsync(tau, tj, size_t(b->M) * 8, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && j) e = cudaMemcpyAsync(j, tj + b->M, size_t(3) * b->M * 8, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(tj);
    if (e != cudaSuccess) return fail(c, WSLDA_ECUDA, std::string("tau/j: ") + cudaGetErrorString(e));
    collect_profile(c);
  }
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return WSLDA_OK;
}

wslda_status wslda_get_spin_densities(wslda_ctx* c, int box, double* rho_a, double* rho_b, double* nu,
                                      double* tau_a, double* tau_b, double* j_a, double* j_b) {
  CHECK_CTX(c);
  Box* b = get_box(c, box);
  if (!b || !b->aslda) return fail(c, WSLDA_EINVAL, "get_spin_densities: bad box or not an ASLDA box");
  if (!b->loaded) return fail(c, WSLDA_ESTATE, "get_spin_densities before load_states");
  if (!c->started) {
    wslda_status st = refresh_fields(c, *b, b->iphi, 1);
    if (st) return st;
  }
  const size_t M = size_t(b->M);
  const std::pair<double*, const double*> cp[4] = {{rho_a, b->rho}, {rho_b, b->rho_b}, {tau_a, b->tauj},
                                                   {tau_b, b->tauj_b}};
  for (int i = 0; i < 4; ++i)
    if (cp[i].first) CUDA_TRY(c, cudaMemcpyAsync(cp[i].first, cp[i].second, M * 8, cudaMemcpyDeviceToHost, c->stream));
  if (nu) CUDA_TRY(c, cudaMemcpyAsync(nu, b->nu, M * 16, cudaMemcpyDeviceToHost, c->stream));
  if (j_a) CUDA_TRY(c, cudaMemcpyAsync(j_a, b->tauj + M, 3 * M * 8, cudaMemcpyDeviceToHost, c->stream));
  if (j_b) CUDA_TRY(c, cudaMemcpyAsync(j_b, b->tauj_b + M, 3 * M * 8, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return WSLDA_OK;
}

wslda_status wslda_get_spin_fields(wslda_ctx* c, int box, double* V_a, double* V_b, double* delta) {
  CHECK_CTX(c);
  Box* b = get_box(c, box);
  if (!b || !b->aslda) return fail(c, WSLDA_EINVAL, "get_spin_fields: bad box or not an ASLDA box");
  if (!b->loaded) return fail(c, WSLDA_ESTATE, "get_spin_fields before load_states");
  if (!c->started) {
    wslda_status st = refresh_fields(c, *b, b->iphi, 1);
    if (st) return st;
  }
  const size_t M = size_t(b->M);
  if (V_a) CUDA_TRY(c, cudaMemcpyAsync(V_a, b->U, M * 8, cudaMemcpyDeviceToHost, c->stream));
  if (V_b) CUDA_TRY(c, cudaMemcpyAsync(V_b, b->U_b, M * 8, cudaMemcpyDeviceToHost, c->stream));
  if (delta) CUDA_TRY(c, cudaMemcpyAsync(delta, b->delta, M * 16, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return WSLDA_OK;
}

wslda_status wslda_get_fields(wslda_ctx* c, int box, double* U, double* delta) {
  CHECK_CTX(c);
  Box* b = get_box(c, box);
  if (!b) return fail(c, WSLDA_EINVAL, "get_fields: bad box");
  if (!b->loaded) return fail(c, WSLDA_ESTATE, "get_fields before load_states");
  if (!c->started) {
    wslda_status st = refresh_fields(c, *b, b->iphi, 1);
    if (st) return st;
  }
  if (U) CUDA_TRY(c, cudaMemcpyAsync(U, b->U, size_t(b->M) * 8, cudaMemcpyDeviceToHost, c->stream));
  if (delta) CUDA_TRY(c, cudaMemcpyAsync(delta, b->delta, size_t(b->M) * 16, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return WSLDA_OK;
}

wslda_status wslda_get_energy(wslda_ctx* c, int box, wslda_energy* out) {
  CHECK_CTX(c);
  Box* b = get_box(c, box);
  if (!b || !out) return fail(c, WSLDA_EINVAL, "get_energy: bad box or null pointer");
  if (!b->loaded) return fail(c, WSLDA_ESTATE, "get_energy before load_states");
  wslda_status st;
  if (!c->started && (st = refresh_fields(c, *b, b->iphi, 1))) return st;
  double h[16];
  st = c->prec == WSLDA_MIXED ? compute_energy<float>(c, *b, h) : compute_energy<double>(c, *b, h);
  if (st) return st;
  collect_profile(c);
  out->e_kin = h[0];
  out->e_pot = h[1];
  out->e_pair = h[2];
  out->e_ext = h[3];
  out->e_pair_ext = h[4];
  out->e_total = h[5];
  out->n_part = h[6];
  out->e_cur = h[7];
  return WSLDA_OK;
}

wslda_status wslda_eval_f(wslda_ctx* c, int box, double* f) {
  CHECK_CTX(c);
  Box* b = get_box(c, box);
  if (!b || (!f && b->n > 0)) return fail(c, WSLDA_EINVAL, "eval_f: bad box or null pointer");
  if (!b->loaded) return fail(c, WSLDA_ESTATE, "eval_f before load_states");
  if (c->started) return fail(c, WSLDA_ESTATE, "eval_f is a diagnostic of the loaded states, before wslda_start");
  wslda_status st;
  if ((st = refresh_fields(c, *b, b->iphi, 1))) return st;
  const int out = b->ih[0];
  st = c->prec == WSLDA_MIXED ? eval_f_into<float>(c, *b, b->iphi, out) : eval_f_into<double>(c, *b, b->iphi, out);
  if (st) return st;
  std::swap(b->iphi, b->ih[0]);
  st = wslda_get_states(c, box, f, 0);
  std::swap(b->iphi, b->ih[0]);
  if (st) return st;
  collect_profile(c);
  return check_device_error(c);
}

wslda_status wslda_get_variant(wslda_ctx* c, int box, char* desc, int len) {
  CHECK_CTX(c);
  Box* b = get_box(c, box);
  if (!b || !desc || len <= 0) return fail(c, WSLDA_EINVAL, "get_variant: bad arguments");
  const KernelSet* y = b->ks_y ? b->ks_y : b->ks;
  snprintf(desc, size_t(len),
           "cluster=%d threads=%d lanes_per_pencil=%d,%d,%d ctas_per_sm=%d smem=%zu persistent_clusters=%d; "
           "stage Y: cluster=%d threads=%d lanes_per_pencil=%d,%d,%d ctas_per_sm=%d persistent_clusters=%d",
           b->ks->cs, b->ks->bt, b->ks->tx, b->ks->ty, b->ks->tz, b->ks->minb, b->ks->smem, b->ncl, y->cs, y->bt,
           y->tx, y->ty, y->tz, y->minb, b->ks_y ? b->ncl_y : b->ncl);
  return WSLDA_OK;
}

wslda_status wslda_check_conservation(wslda_ctx* c, int box, double e_tol, double n_tol, double* de, double* dn) {
  CHECK_CTX(c);
  Box* b = get_box(c, box);
  if (!b) return fail(c, WSLDA_EINVAL, "check_conservation: bad box");
  if (!c->started) return fail(c, WSLDA_ESTATE, "check_conservation before wslda_start");
  double h[16];
  wslda_status st = c->prec == WSLDA_MIXED ? compute_energy<float>(c, *b, h) : compute_energy<double>(c, *b, h);
  if (st) return st;
  const double e = conserved_energy(*b, h);
  const double rel_e = std::fabs(e - b->e0) / std::max(std::fabs(b->e0), 1e-300);
  const double rel_n = std::fabs(h[6] - b->n0) / std::max(std::fabs(b->n0), 1e-300);
  if (de) *de = rel_e;
  if (dn) *dn = rel_n;
  if (!(rel_e <= e_tol) || !(rel_n <= n_tol))
    return fail(c, WSLDA_EDRIFT, "conservation check: relative energy drift " + std::to_string(rel_e) +
                                     ", particle-number drift " + std::to_string(rel_n));
  return WSLDA_OK;
}

wslda_status wslda_set_graph(wslda_ctx* c, int enable, int nstreams) {
  CHECK_CTX(c);
  drop_graphs(c);
  c->use_graph = enable != 0;
  if (c->use_graph && c->side.empty()) {
    const int k = std::max(1, std::min(nstreams > 0 ? nstreams : 4, 16));
    CUDA_TRY(c, cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
    CUDA_TRY(c, cudaEventCreateWithFlags(&c->cap_in, cudaEventDisableTiming));
    CUDA_TRY(c, cudaEventCreateWithFlags(&c->cap_out, cudaEventDisableTiming));
    CUDA_TRY(c, cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming));
    for (int i = 0; i < k; ++i) {
      cudaStream_t s = nullptr;
      cudaEvent_t e = nullptr;
      CUDA_TRY(c, cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
      CUDA_TRY(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      c->side.push_back(s);
      c->join_ev.push_back(e);
    }
  }
  return WSLDA_OK;
}

wslda_status wslda_get_time(wslda_ctx* c, double* t, int64_t* steps) {
  CHECK_CTX(c);
  if (t) *t = c->t;
  if (steps) *steps = c->steps;
  return WSLDA_OK;
}

int64_t wslda_memory_bytes(const wslda_ctx* c) { return c ? c->bytes : 0; }

wslda_status wslda_set_profiling(wslda_ctx* c, int enable) {
  CHECK_CTX(c);
  collect_profile(c);
  c->prof = enable != 0;
  for (int i = 0; i < NPROF; ++i) {
    c->prof_ms[i] = 0.0;
    c->prof_n[i] = 0;
  }
  return WSLDA_OK;
}

int64_t wslda_launch_count(const wslda_ctx* c) { return c ? c->launches : 0; }

wslda_status wslda_get_kernel_time(wslda_ctx* c, int kind, double* total_ms, int64_t* launches) {
  CHECK_CTX(c);
  if (kind < 0 || kind >= NPROF) return fail(c, WSLDA_EINVAL, "kernel kind out of range");
  collect_profile(c);
  if (total_ms) *total_ms = c->prof_ms[kind];
  if (launches) *launches = c->prof_n[kind];
  return WSLDA_OK;
}

// File layout: "WSLDATD1", prec, nboxes, t, steps, dt_start, started; per box:
// nx ny nz n iphi ih[4], then for each of the 5 slots its states and per-state
// scale, then lam, vext, dext, wm, wp.
wslda_status wslda_save(wslda_ctx* c, const char* path) {
  CHECK_CTX(c);
  if (!path) return fail(c, WSLDA_EINVAL, "save: null path");
  FILE* f = fopen(path, "wb");
  if (!f) return fail(c, WSLDA_EINVAL, std::string("save: cannot open ") + path);
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  const char magic[8] = {'W', 'S', 'L', 'D', 'A', 'T', 'D', '4'};
  int32_t hdr[3] = {c->prec, int32_t(c->boxes.size()), c->started ? 1 : 0};
  fwrite(magic, 1, 8, f);
  fwrite(hdr, sizeof(hdr), 1, f);
  fwrite(&c->t, 8, 1, f);
  fwrite(&c->steps, 8, 1, f);
  fwrite(&c->dt_start, 8, 1, f);
  std::vector<char> host;
  auto dump = [&](const void* d, size_t bytes) -> bool {
    host.resize(bytes);
    if (cudaMemcpy(host.data(), d, bytes, cudaMemcpyDeviceToHost) != cudaSuccess) return false;
    return fwrite(host.data(), 1, bytes, f) == bytes;
  };
  bool ok = true;
  for (Box& b : c->boxes) {
    // the launch variant travels with the state, so that a resumed run uses the
    // same kernels (different variants round differently)
    const KernelSet* ky = b.ks_y ? b.ks_y : b.ks;
    const int ny = b.ks_y ? b.ncl_y : b.ncl;
    int64_t bh[25] = {b.lat.nx, b.lat.ny, b.lat.nz, b.n, b.D, b.iphi, b.ih[0], b.ih[1], b.ih[2], b.ih[3], b.ih[4],
                      b.ks->cs, b.ks->bt, b.ks->tx, b.ks->ty, b.ks->tz, b.ks->minb, b.ncl > 0 ? 1 : 0,
                      ky->cs, ky->bt, ky->tx, ky->ty, ky->tz, ky->minb, ny > 0 ? 1 : 0};
    fwrite(bh, sizeof(bh), 1, f);
    const size_t sb = size_t(b.n) * 2 * b.M * b.csize;
    for (int i = 0; i < b.D + 2 && ok; ++i) ok = dump(b.slot[i], sb) && dump(b.sc[i], std::max<int64_t>(b.n, 1) * 8);
    ok = ok && dump(b.lam, size_t(b.M) * 8) && dump(b.vext, size_t(b.M) * 8) && dump(b.dext, size_t(b.M) * 16) &&
         dump(b.wm, std::max<int64_t>(b.n, 1) * 8) && dump(b.wp, std::max<int64_t>(b.n, 1) * 8);
  }
  fclose(f);
  if (!ok) return fail(c, WSLDA_ECUDA, "save: device read or file write failed");
  return WSLDA_OK;
}

wslda_status wslda_load(wslda_ctx* c, const char* path) {
  CHECK_CTX(c);
  if (!path) return fail(c, WSLDA_EINVAL, "load: null path");
  FILE* f = fopen(path, "rb");
  if (!f) return fail(c, WSLDA_EINVAL, std::string("load: cannot open ") + path);
  char magic[8];
  int32_t hdr[3];
  double t, dts;
  int64_t steps;
  bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, "WSLDATD4", 8) == 0 && fread(hdr, sizeof(hdr), 1, f) == 1 &&
            fread(&t, 8, 1, f) == 1 && fread(&steps, 8, 1, f) == 1 && fread(&dts, 8, 1, f) == 1;
  if (!ok || hdr[0] != c->prec || hdr[1] != int32_t(c->boxes.size())) {
    fclose(f);
    return fail(c, WSLDA_EINVAL, "load: file does not match this context (precision / box count)");
  }
  std::vector<char> host;
  auto slurp = [&](void* d, size_t bytes) -> bool {
    host.resize(bytes);
    if (fread(host.data(), 1, bytes, f) != bytes) return false;
    return cudaMemcpy(d, host.data(), bytes, cudaMemcpyHostToDevice) == cudaSuccess;
  };
  for (Box& b : c->boxes) {
    int64_t bh[25];
    ok = ok && fread(bh, sizeof(bh), 1, f) == 1 && bh[0] == b.lat.nx && bh[1] == b.lat.ny && bh[2] == b.lat.nz &&
         bh[3] == b.n && bh[4] == b.D;
    if (!ok) break;
    b.iphi = int(bh[5]);
    for (int i = 0; i < 5; ++i) b.ih[i] = int(bh[6 + i]);
    for (int stage = 0; stage < 2; ++stage) {
      const int64_t* id = bh + 11 + 7 * stage;
      for (const KernelSet& k : registry())
        if (k.prec == (c->prec == WSLDA_MIXED ? 1 : 0) && k.nx == b.lat.nx && k.ny == b.lat.ny &&
            k.nz == b.lat.nz && k.cs == id[0] && k.bt == id[1] && k.tx == id[2] && k.ty == id[3] && k.tz == id[4] &&
            k.minb == id[5]) {
          (stage ? b.ks_y : b.ks) = &k;
          (stage ? b.ncl_y : b.ncl) = id[6] ? resident_clusters(&k) : 0;
          break;
        }
    }
    const size_t sb = size_t(b.n) * 2 * b.M * b.csize;
    for (int i = 0; i < b.D + 2 && ok; ++i) ok = slurp(b.slot[i], sb) && slurp(b.sc[i], std::max<int64_t>(b.n, 1) * 8);
    ok = ok && slurp(b.lam, size_t(b.M) * 8) && slurp(b.vext, size_t(b.M) * 8) && slurp(b.dext, size_t(b.M) * 16) &&
         slurp(b.wm, std::max<int64_t>(b.n, 1) * 8) && slurp(b.wp, std::max<int64_t>(b.n, 1) * 8);
    if (!ok) break;
    if (c->prec == WSLDA_MIXED) {
      launch_to_real<float>(b.wm, static_cast<float*>(b.wm_r), std::max<int64_t>(b.n, 1), c->stream);
      launch_to_real<float>(b.wp, static_cast<float*>(b.wp_r), std::max<int64_t>(b.n, 1), c->stream);
    } else {
      cudaMemcpyAsync(b.wm_r, b.wm, std::max<int64_t>(b.n, 1) * 8, cudaMemcpyDeviceToDevice, c->stream);
      cudaMemcpyAsync(b.wp_r, b.wp, std::max<int64_t>(b.n, 1) * 8, cudaMemcpyDeviceToDevice, c->stream);
    }
    b.loaded = true;
    wslda_status st = refresh_fields(c, b, b.iphi, 0);
    if (st) {
      fclose(f);
      return st;
    }
  }
  fclose(f);
  if (!ok) return fail(c, WSLDA_EINVAL, "load: truncated or mismatched file");
  drop_graphs(c);
  c->t = t;
  c->steps = steps;
  c->dt_start = dts;
  c->started = hdr[2] != 0;
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return WSLDA_OK;
}

}  // extern "C"
