// Internal declarations shared by the host runtime and the kernel instances.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/wslda_td.h"
#include "stage.cuh"

namespace wslda {

// nclusters > 0 launches that many clusters, each looping over states
// cluster, cluster + nclusters, ... (persistent); 0 launches one per state.
using LaunchFn = cudaError_t (*)(const void* args, int nstates, int nclusters, cudaStream_t s);

// One compiled lattice shape / precision: launchers for every stage mode.
struct KernelSet {
  int prec;  // 0 = double, 1 = float (mixed)
  int nx, ny, nz;
  int cs, bt, tx, ty, tz, minb;
  size_t smem;
  LaunchFn launch[NMODES];
  // the modes that apply H, compiled for the general functional (current
  // term, per-site alpha; one cluster per state); NULL for the other modes
  LaunchFn launch_gen[NMODES];
  const void* fn[NMODES];
};

std::vector<KernelSet>& registry();

struct Registrar {
  explicit Registrar(const KernelSet& k) { registry().push_back(k); }
};

template <class G, int MODE, bool PERSIST, bool GEN = false>
cudaError_t launch_stage_as(const StageArgs<typename G::R>& a, int ncl, cudaStream_t s) {
  auto kern = stage_kernel<G, MODE, PERSIST, GEN>;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(G::smem_bytes));
    if (e != cudaSuccess) return e;
    if (G::CS > 8) {
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) return e;
    }
    configured = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(ncl) * G::CS);
  cfg.blockDim = dim3(G::BT);
  cfg.dynamicSmemBytes = G::smem_bytes;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = G::CS;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a);
}

template <class G, int MODE>
cudaError_t launch_stage(const void* args, int nstates, int nclusters, cudaStream_t s) {
  StageArgs<typename G::R> a = *static_cast<const StageArgs<typename G::R>*>(args);
  a.nstates = nstates;
  if (nclusters > 0 && nclusters < nstates) return launch_stage_as<G, MODE, true>(a, nclusters, s);
  return launch_stage_as<G, MODE, false>(a, nstates, s);
}
// general-functional instance: always one cluster per state
template <class G, int MODE>
cudaError_t launch_stage_gen(const void* args, int nstates, int, cudaStream_t s) {
  StageArgs<typename G::R> a = *static_cast<const StageArgs<typename G::R>*>(args);
  a.nstates = nstates;
  return launch_stage_as<G, MODE, false, true>(a, nstates, s);
}

template <class G>
KernelSet make_set() {
  KernelSet k;
  k.prec = sizeof(typename G::R) == 4 ? 1 : 0;
  k.nx = G::NX; k.ny = G::NY; k.nz = G::NZ;
  k.cs = G::CS; k.bt = G::BT; k.tx = G::TX; k.ty = G::TY; k.tz = G::TZ; k.minb = G::MINB;
  k.smem = G::smem_bytes;
  k.launch[MODE_X] = launch_stage<G, MODE_X>;
  k.launch[MODE_Y] = launch_stage<G, MODE_Y>;
  k.launch[MODE_F] = launch_stage<G, MODE_F>;
  k.launch[MODE_HORNER] = launch_stage<G, MODE_HORNER>;
  k.launch[MODE_EKIN] = launch_stage<G, MODE_EKIN>;
  k.launch[MODE_GRAD] = launch_stage<G, MODE_GRAD>;
  k.launch[MODE_X3] = launch_stage<G, MODE_X3>;
  k.launch[MODE_X5] = launch_stage<G, MODE_X5>;
  k.launch[MODE_LAP] = launch_stage<G, MODE_LAP>;
  k.launch[MODE_AGRAD] = launch_stage<G, MODE_AGRAD>;
  k.launch[MODE_KALPHA] = launch_stage<G, MODE_KALPHA>;
  for (int m = 0; m < NMODES; ++m) k.launch_gen[m] = nullptr;
  k.launch_gen[MODE_X] = launch_stage_gen<G, MODE_X>;
  k.launch_gen[MODE_Y] = launch_stage_gen<G, MODE_Y>;
  k.launch_gen[MODE_F] = launch_stage_gen<G, MODE_F>;
  k.launch_gen[MODE_HORNER] = launch_stage_gen<G, MODE_HORNER>;
  k.launch_gen[MODE_X3] = launch_stage_gen<G, MODE_X3>;
  k.launch_gen[MODE_X5] = launch_stage_gen<G, MODE_X5>;
  k.fn[MODE_X] = (const void*)stage_kernel<G, MODE_X, false>;
  k.fn[MODE_Y] = (const void*)stage_kernel<G, MODE_Y, false>;
  k.fn[MODE_F] = (const void*)stage_kernel<G, MODE_F, false>;
  k.fn[MODE_HORNER] = (const void*)stage_kernel<G, MODE_HORNER, false>;
  k.fn[MODE_EKIN] = (const void*)stage_kernel<G, MODE_EKIN, false>;
  k.fn[MODE_GRAD] = (const void*)stage_kernel<G, MODE_GRAD, false>;
  k.fn[MODE_X3] = (const void*)stage_kernel<G, MODE_X3, false>;
  k.fn[MODE_X5] = (const void*)stage_kernel<G, MODE_X5, false>;
  k.fn[MODE_LAP] = (const void*)stage_kernel<G, MODE_LAP, false>;
  k.fn[MODE_AGRAD] = (const void*)stage_kernel<G, MODE_AGRAD, false>;
  k.fn[MODE_KALPHA] = (const void*)stage_kernel<G, MODE_KALPHA, false>;
  return k;
}

#define WSLDA_CAT2(a, b) a##b
#define WSLDA_CAT(a, b) WSLDA_CAT2(a, b)
// WSLDA_INSTANCE(real type, NX, NY, NZ, cluster size, threads, lanes per x/y/z pencil)
// optional last argument: CTAs per SM the register budget is sized for
#define WSLDA_INSTANCE(R, NX, NY, NZ, CS, BT, TX, TY, TZ, ...)                              \
  static ::wslda::Registrar WSLDA_CAT(wslda_reg_, __COUNTER__)(                            \
      ::wslda::make_set<::wslda::Geometry<R, NX, NY, NZ, CS, BT, TX, TY, TZ, ##__VA_ARGS__>>());

// ---------------------------------------------------------------------------
// Site-major kernels (densities.cu)
// ---------------------------------------------------------------------------
struct FunctionalDev {
  int kind;  // 0 slda, 1 bdg
  double B, C, inv_4pi_a, mu, ec, rho_floor;
  double A;  // inverse effective mass (1 unless the box carries the current terms)
};

// Partial sums over chunks of states: part[c][0..2][M] = rho, Re nu, Im nu.
// Stored states are scaled by sc[n] (deferred normalisation).
template <typename R>
cudaError_t launch_density_partial(const cx<R>* phi, const double* sc, const R* wm, const R* wp, int64_t nstates,
                                   int M, int nchunk, int64_t chunk, double* part, cudaStream_t s);

// Quantum friction (Sec. 5.2.4) added to the H fields in place:
// W += -(alpha / rho0) div_j,  D += Delta [beta sin(arg nu - arg B') + i gamma (N - N_req) / N_req],
// N = dV sum 2 rho_sigma (one CTA: the sum, then the update).
template <typename R>
cudaError_t launch_apply_friction(int M, double dV, double alpha, double beta, double gamma, double rho0,
                                  double n_req, const double* rho, const double* nu, const double* delta,
                                  const double* divj, const double* bp3, fx4<R>* WD, cudaStream_t s);

// Number of state chunks of the density reduction for M sites and n states.
int density_chunks(int M, int64_t nstates, int is_float);

// Sum the chunk partials, build (U, Delta) with the frozen regulator lam
// (or first compute lam by the t = 0 fixed point when init_lam), and write
// the H fields in precision R.
template <typename R>
cudaError_t launch_potentials(const double* part, int nchunk, int M, FunctionalDev fn, const double* vext,
                              const double* dext, double* lam, int init_lam, const double* j, double* rho, double* nu,
                              double* U, double* delta, fx4<R>* WD, cudaStream_t s);

// Current potential of A != 1 boxes: AV[s] = {A_x, A_y, A_z, div A / 2} with
// A_d = (1 - A) j_d / max(rho_s, rho_floor); d1 = first columns of the
// per-axis first-derivative matrices, concatenated x, y, z.
template <typename R>
cudaError_t launch_current_fields(int nx, int ny, int nz, double A, double rho_floor, const double* rho,
                                  const double* j, const double* d1, fx4<R>* AV, cudaStream_t s);

// tau and j (Eqs. nab3D..jab3D) from per-state contributions stored as
// [n][2][M] complex {tau, j_x}, {j_y, j_z}: summed over states per site.
template <typename R>
cudaError_t launch_sum_tauj(const cx<R>* contrib, int64_t nstates, int M, int nchunk, int64_t chunk, double* part,
                            double* tau, double* j, cudaStream_t s);

// Deferred normalisation: sc[i] = 1/sqrt(dV sum_{r<cs} npart[16 i + r]).
cudaError_t launch_finalize_norm(const double* npart, int cs, int64_t n, double dV, double* sc, int* err,
                                 cudaStream_t s);

// Energy terms (Sec. 3.2) from the site fields and per-state kinetic values.
cudaError_t launch_energy(int M, int64_t nstates, FunctionalDev fn, const double* rho, const double* nu,
                          const double* delta, const double* vext, const double* dext, const double* ekin2,
                          const double* wm, const double* wp, const double* j, double dV, double* out8,
                          cudaStream_t s);

// Spin-imbalanced ASLDA (aslda.cu): per-site potentials from the u-part and
// v-part density partials and {tau, j} of each species, then the fields of H
// that need neighbouring sites (lap alpha, div A), and the energy terms.
cudaError_t launch_aslda_potentials(const double* part_a, const double* part_b, int nchunk, int M, const double* tj_a,
                                    const double* tj_b, const double* vext, double mu_a, double mu_b, double C,
                                    double ec, double rho_floor, double* lam, int init_lam, double* rho_a,
                                    double* rho_b, double* nu, double* Va, double* Vb, double* delta, double* af,
                                    cudaStream_t s);
template <typename R>
cudaError_t launch_aslda_fields(int nx, int ny, int nz, const double* af, const double* Va, const double* Vb,
                                const double* delta, const double* vext, const double* dext, double mu_a, double mu_b,
                                const double* d1, const double* d2, fx4<R>* WD, cx<R>* alf, fx4<R>* av_a,
                                fx4<R>* av_b, cudaStream_t s);
cudaError_t launch_aslda_energy(int M, const double* rho_a, const double* rho_b, const double* nu, const double* tj_a,
                                const double* tj_b, const double* lam, const double* vext, const double* dext, double C,
                                double rho_floor, double dV, double* out8, cudaStream_t s);

// Plane-wave states of a uniform solution (uniform.cu); dst is float2 or double2.
cudaError_t launch_fill_plane_waves(void* dst, int is_float, const wslda_lattice& lat, double mu_eff, double delta,
                                    const int64_t* kidx_dev, int64_t n, int partners, cudaStream_t s);

// Static self-consistent solve (scf.cu): the box buffers it reads and writes.
struct ScfBox {
  wslda_lattice lat;
  FunctionalDev fn;
  int M;
  int prec;
  void* states;  // [M][2][M] complex slot receiving the eigenstates
  double* sc;    // that slot's per-state scale, set to 1
  const double* vext;
  const double* dext;  // zero
  double *rho, *nu, *delta, *ekin2, *wm, *wp, *out8;
  cudaStream_t s;
};
wslda_status static_solve(const ScfBox& b, const double* U0, const double* D0, const wslda_scf_params& p,
                          double* qpE, wslda_scf_result* res, std::string& err);

template <typename R>
cudaError_t launch_narrow(const double* src, cx<R>* dst, int64_t ncomplex, int* err, cudaStream_t s);
template <typename R>
cudaError_t launch_widen(const cx<R>* src, double* dst, int64_t ncomplex, const double* sc, int64_t first,
                         int64_t per_state, cudaStream_t s);
cudaError_t launch_fill(double* p, double v, int64_t n, cudaStream_t s);
// Component comp (0 = u, 1 = v) of every state times phase[r] ([M] complex double).
template <typename R>
cudaError_t launch_imprint(cx<R>* states, int64_t nstates, int M, int comp, const double* phase, cudaStream_t s);
// dst = sc[state] * src (sc NULL: 1), complex float <-> double; non-finite src sets err bit 1.
template <typename S, typename D>
cudaError_t launch_rescale(const S* src, D* dst, int64_t n, const double* sc, int64_t first, int64_t per_state,
                           int* err, cudaStream_t s);
template <typename R>
cudaError_t launch_to_real(const double* src, R* dst, int64_t n, cudaStream_t s);

}  // namespace wslda
