/*
 * wslda_td.h -- C ABI of the B300 time-dependent SLDA (TDSLDA) library.
 *
 * The library advances every quasiparticle pair (u_n, v_n) of one or more
 * periodic 3D boxes with the modified equation of motion
 *     i d(phi_n)/dt = [H - <H>_n] phi_n                (Sec. 3.3, Eq. shorttdproblem-mod)
 * using the AB4AM5 predictor-corrector of Alg. 2, the kinetic term through
 * FFTs (Eq. derivative-spectral, A_sigma = 1 so only the Laplacian, Eq. h_sigma_A1),
 * the densities rho, nu summed over all states (Eqs. nab3D..jab3D, spin
 * symmetric, frozen thermal weights Sec. 2.5) and the potentials rebuilt from
 * the SLDA or BdG functional with the regularised coupling of Eq. Creg.
 *
 * Conventions shared by every call
 *  - Units m = hbar = 1 (Sec. 2.1). Lattice sites are flattened as
 *    (ix * ny + iy) * nz + iz (x slowest, z fastest), M = nx * ny * nz.
 *  - A set of states is stored as [n][2][M] complex numbers, component 0 = u,
 *    component 1 = v, each complex as two doubles (re, im), normalised to
 *    sum_r dV (|u|^2 + |v|^2) = 1.
 *  - Complex fields ([M] complex) are interleaved (re, im) doubles.
 *  - Ownership: the caller owns every buffer it passes; the library copies
 *    in and out and keeps no pointer after a call returns. Device pointers
 *    (on_device = 1) must be device memory of the context's device; they are
 *    read or written on the context's stream and the call synchronises that
 *    stream before returning.
 *  - Errors: every call returns a wslda_status; nothing aborts or throws
 *    across the ABI. The first failure is sticky on the context (later calls
 *    return WSLDA_ESTATE) and wslda_last_error() describes it.
 *  - Precision: WSLDA_FP64 keeps states, FFTs and all arithmetic in double.
 *    WSLDA_MIXED stores states as complex float, runs FFTs, the Hamiltonian
 *    and the integrator combinations in float, and accumulates densities,
 *    norms and energies in double through compensated float partial sums;
 *    potentials and the regulator are double. Inputs and outputs of the ABI
 *    are always double.
 */
#ifndef WSLDA_TD_H
#define WSLDA_TD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wslda_ctx wslda_ctx;

typedef enum {
  WSLDA_OK = 0,
  WSLDA_EINVAL = 1,      /* bad argument (sizes, null pointers, dt = 0, ...) */
  WSLDA_ENOMEM = 2,      /* device memory budget exceeded; nothing was allocated */
  WSLDA_ECUDA = 3,       /* a CUDA runtime call failed */
  WSLDA_ENAN = 4,        /* a non-finite value in an input or a state norm */
  WSLDA_EDRIFT = 5,      /* conservation check exceeded its tolerance */
  WSLDA_ETIMEOUT = 6,    /* a bounded device-side wait gave up */
  WSLDA_ESTATE = 7,      /* call out of order, or the context holds an earlier error */
  WSLDA_EUNSUPPORTED = 8 /* lattice shape / precision without a compiled kernel */
} wslda_status;

typedef enum { WSLDA_FP64 = 0, WSLDA_MIXED = 1 } wslda_precision;

typedef enum {
  WSLDA_FUNC_SLDA_A1 = 0, /* SLDA with A forced to 1 (Sec. 2.4, last paragraph) */
  WSLDA_FUNC_BDG = 1,     /* BdG: A = 1, B = 0, coupling 4 pi a (Eq. HBdG) */
  WSLDA_FUNC_SLDA = 2,    /* SLDA-type with a constant A (field A), current terms included */
  WSLDA_FUNC_ASLDA = 3    /* spin-imbalanced ASLDA (Sec. 2.4): A_a(p), A_b(p), B(p) printed, C given */
} wslda_functional_kind;

/* Periodic lattice (Sec. 3.1). Every n must be even; see
 * wslda_lattice_supported() for the shapes with compiled kernels. */
typedef struct {
  int nx, ny, nz;
  double dx, dy, dz;
} wslda_lattice;

/* Energy density functional and its regularised coupling (Sec. 2.4, 2.6).
 *  slda_a1: E_0 = (tau_a + tau_b)/2 + 3/5 B rho eF(rho) + g_eff |nu|^2,
 *        1/g_eff = rho^(1/3)/C - Lambda_c,  U = B eF - |Delta|^2/(3 C rho^(2/3))
 *  slda (constant A, spin-symmetric; the ASLDA functional at p = 0 has
 *        A = 1.094): E_0 + E_CM adds sum_s [(A - 1) tau_s / 2 + (1 - A) j_s^2 / (2 rho_s)]
 *        (Eqs. sldae-functional-generic..sldae-functional), so that
 *        h = -A/2 lap + U + V_ext - (i/2){A_s, grad} (Eq. h_sigma) with the
 *        current potential A_s = (1 - A) j_s / rho_s and
 *        U += (A - 1) j_s^2 / (2 rho_s^2); Lambda_c uses A_+ = A. j_s is
 *        reduced over all states at every stage (Eq. jab3D); rho_s is floored
 *        at rho_floor in these terms. A = 1 gives slda_a1. Static solves and
 *        the dissipative terms are not available for it (WSLDA_EUNSUPPORTED).
 *  bdg : 1/g_eff = inv_4pi_a - Lambda_c,     U = 0
 *  aslda (spin-imbalanced, Secs. 2.3-2.4): the states are those of Eq. HpsiEpsi
 *        over the whole spectrum, phi_n = (u_{n,a}, v_{n,b}) with the weights
 *        w_plus = f(E_n) for u and w_minus = f(-E_n) for v; densities of
 *        Eqs. na3D..jb3D (rho_a = sum f(E)|u|^2, rho_b = sum f(-E)|v|^2,
 *        nu = 1/2 sum (f(-E) - f(E)) u v^*, tau_s and j_s the same way with
 *        Nyquist-free gradients), all reduced at every stage; A_a(p) = A_b(-p)
 *        and B(p) as printed, p = (rho_a - rho_b)/(rho_a + rho_b), C = C
 *        (the ASLDA value is -11.11); potentials V_s = dE/d rho_s (with the
 *        p-derivative terms), alpha_s = A_s(p), current potentials
 *        (1 - A_s) j_s / rho_s; the kinetic operator -1/2 grad.alpha_s grad of
 *        Eq. kinop-alpha; mu = mu_a on the u row, mu_b on the v row; one V_ext
 *        for both species; Lambda_c with the spin averages of Sec. 2.6. B and
 *        A are not read. Static solves and the dissipative terms are not
 *        available for it (WSLDA_EUNSUPPORTED).
 *  Delta = -g_eff nu (Eq. Delta). mu is the chemical potential on the diagonal
 *  of H. ec <= 0 selects the zone-corner cutoff (pi^2/2)(1/dx^2+1/dy^2+1/dz^2).
 *  rho_floor bounds rho from below inside the potentials only. A is read for
 *  kind slda only, mu_b for kind aslda only. */
typedef struct {
  int kind;
  double B, C;
  double inv_4pi_a;
  double mu;
  double ec;
  double rho_floor;
  double A;
  double mu_b;
} wslda_functional;

/* Energy terms of Sec. 3.2. e_kin is A times the sum of the kinetic
 * densities; e_cur = int sum_s (1 - A) j_s^2 / (2 rho_s) (kind slda, else 0).
 * e_total is the sum of the terms; the evolution conserves e_total - mu * n_part
 * (Eq. E_tot). */
typedef struct {
  double e_kin, e_pot, e_pair, e_ext, e_pair_ext, e_total, n_part, e_cur;
} wslda_energy;

/* Create a context on the current CUDA device. `cuda_stream` is a borrowed
 * cudaStream_t (NULL = legacy default stream) on which all work is queued. */
wslda_status wslda_create(int precision, void* cuda_stream, wslda_ctx** out);
void wslda_destroy(wslda_ctx* ctx);
const char* wslda_last_error(const wslda_ctx* ctx);

/* 1 if kernels for this lattice shape and precision are compiled in. */
int wslda_lattice_supported(int precision, int nx, int ny, int nz);
/* Number of compiled launch variants for the shape (0 if unsupported); the
 * environment variable WSLDA_VARIANT=<index> forces one of them (with
 * WSLDA_PERSIST=0/1 fixing the launch form, WSLDA_VARIANT_Y=<index> then puts
 * the corrector stage on another variant). */
int wslda_lattice_variants(int precision, int nx, int ny, int nz);

/* Predictor-corrector scheme of the boxes added afterwards (Sec. 3.3):
 * AB4AM5 (default, Alg. 2, five state buffers), AB3AM4 (four buffers,
 * fourth order) or AB5AM5 (six buffers, fifth order with a fifth-order
 * predictor). Each is run in place in the manner of Alg. 2: the predictor
 * stage writes f(phi), the predictor and the corrector partial (over the
 * oldest history value, its last use); the start-up takes p - 1 Taylor steps
 * for a predictor of order p. WSLDA_ESTATE once a box exists. */
typedef enum { WSLDA_AB4AM5 = 0, WSLDA_AB3AM4 = 1, WSLDA_AB5AM5 = 2 } wslda_scheme;
wslda_status wslda_set_integrator(wslda_ctx* ctx, int scheme);

/* Add a box with `nstates` quasiparticle states. Allocates its state buffers
 * (phi and the ABM history slots: five for AB4AM5, Alg. 2) after checking the
 * device budget. Returns the box id (>= 0) or -(wslda_status) on failure. */
int wslda_add_box(wslda_ctx* ctx, const wslda_lattice* lat, const wslda_functional* fn, int64_t nstates);

/* External potential V_ext [M] and external pairing field Delta_ext [M complex]
 * (Eq. E_tot, Eq. HpsiEpsi). Both default to zero. */
wslda_status wslda_set_vext(wslda_ctx* ctx, int box, const double* vext, int on_device);
wslda_status wslda_set_dext(wslda_ctx* ctx, int box, const double* dext, int on_device);

/* Dissipative ("quantum friction") terms of Sec. 5.2.4 for one box, added to
 * the fields of H at every evaluation (also during the start-up):
 *   U_diss = -(alpha / rho0) div j_sigma,
 *   Delta_diss = Delta [beta sin(arg nu - arg B') + i gamma (N - n_req) / n_req],
 *   B' = -1/2 sum_n (w-_n - w+_n) (u_n lap v_n^* + v_n^* lap u_n),
 * with div j_sigma = sum_n [w-_n Im(v_n lap v_n^*) - w+_n Im(u_n lap u_n^*)]
 * (the product rule, with the Laplacian of H), N = int (rho_a + rho_b), and
 * Delta the mean-field pairing (without Delta_ext). The energy diagnostics
 * keep the conservative functional. Each evaluation adds one transform pass
 * over the states and a state-sized scratch buffer, allocated on the first
 * call (WSLDA_ENOMEM when it does not fit). All coefficients 0 switch the
 * terms off. rho0, n_req > 0. May be called at any time (captured graphs are
 * dropped). */
wslda_status wslda_set_friction(wslda_ctx* ctx, int box, double alpha, double beta, double gamma, double rho0,
                                double n_req);

/* Load states [n][2][M] complex. w_minus / w_plus are the frozen weights
 * f_beta(-E_n), f_beta(E_n) (Sec. 2.5) as [n] host doubles, or NULL for T = 0
 * (w_minus = 1, w_plus = 0). The mixed path rounds the states to complex float.
 * Non-finite input gives WSLDA_ENAN. */
wslda_status wslda_load_states(wslda_ctx* ctx, int box, const double* uv, const double* w_minus,
                               const double* w_plus, int on_device);

/* Prepare the integrator for every box (Sec. 3.3, start-up). Computes the
 * densities, freezes the regulator Lambda_c at its t = 0 value, then either
 * assumes a stationary state (stationary = 1: the older history is zero) or
 * runs Taylor predictor-corrector steps of order 5 (Eq. Taylor-exp): three for
 * AB4AM5 (two for AB3AM4, four for AB5AM5), which advance the time by that
 * many dt. Must be called again after changing the sign of dt. */
wslda_status wslda_start(wslda_ctx* ctx, int stationary, double dt);

/* Advance every box by nsteps predictor-corrector steps of size dt (Alg. 2
 * for AB4AM5). */
wslda_status wslda_step(wslda_ctx* ctx, double dt, int nsteps);

/* Copy the current states out as [n][2][M] complex double. */
wslda_status wslda_get_states(wslda_ctx* ctx, int box, double* uv, int on_device);

/* The same with complex float elements ([n][2][M], (re, im) float pairs):
 * the mixed path moves its states at their stored precision (half the bytes
 * of the double calls; on load they go straight into the state buffer); the
 * FP64 path widens on load and rounds on read-out. */
wslda_status wslda_load_states_f32(wslda_ctx* ctx, int box, const float* uv, const double* w_minus,
                                   const double* w_plus, int on_device);
wslda_status wslda_get_states_f32(wslda_ctx* ctx, int box, float* uv, int on_device);

/* Densities of the current states: rho = rho_a = rho_b [M], nu [M complex];
 * tau [M] and j [3][M] (Eqs. nab3D..jab3D, gradients with the Nyquist mode
 * zeroed) are computed when the pointers are not NULL. Host pointers. */
wslda_status wslda_get_densities(wslda_ctx* ctx, int box, double* rho, double* nu, double* tau, double* j);

/* Per-species densities of an aslda box (host pointers, each nullable):
 * rho_a, rho_b [M], nu [M complex], tau_a, tau_b [M], j_a, j_b [3][M]
 * (Eqs. na3D..jb3D with the box's frozen weights). For other kinds
 * WSLDA_EINVAL. (wslda_get_densities on an aslda box gives rho = (rho_a + rho_b)/2
 * and nu, and no tau or j.) */
wslda_status wslda_get_spin_densities(wslda_ctx* ctx, int box, double* rho_a, double* rho_b, double* nu,
                                      double* tau_a, double* tau_b, double* j_a, double* j_b);

/* Per-species potentials of an aslda box (host pointers, each nullable):
 * V_a, V_b [M] (dE/d rho_s, without V_ext and mu) and Delta [M complex]
 * (without Delta_ext). For other kinds WSLDA_EINVAL. */
wslda_status wslda_get_spin_fields(wslda_ctx* ctx, int box, double* V_a, double* V_b, double* delta);

/* Potentials built from the current densities: U [M] and Delta [M complex]
 * (without Delta_ext). Host pointers. */
wslda_status wslda_get_fields(wslda_ctx* ctx, int box, double* U, double* delta);

/* Energy terms of the current states (Sec. 3.2). */
wslda_status wslda_get_energy(wslda_ctx* ctx, int box, wslda_energy* out);

/* Conservation diagnostics of the TD codes (Sec. 4.5.1): relative drift of
 * E_tot - mu N (Eq. E_tot) and of N since wslda_start, for one box. Returns
 * WSLDA_EDRIFT (sticky, like every error) when either exceeds its tolerance;
 * de / dn (nullable) receive the drifts. */
wslda_status wslda_check_conservation(wslda_ctx* ctx, int box, double e_tol, double n_tol, double* de, double* dn);

/* Diagnostic: f(phi) = -i [H - <H>_n] phi (Eq. ABM-f) of the current states
 * with potentials from their densities, [n][2][M] complex double on the host. */
wslda_status wslda_eval_f(wslda_ctx* ctx, int box, double* f);

/* Save / restore the full integrator state (states, history, regulator,
 * time and step counter, and the stage-kernel launch variant) to a file;
 * resuming is bit-identical when the loading library has that variant. */
wslda_status wslda_save(wslda_ctx* ctx, const char* path);
wslda_status wslda_load(wslda_ctx* ctx, const char* path);

/* Batched execution of many boxes: when enabled, box i of a step runs on
 * forked stream i mod nstreams (nstreams <= 0: 4) so that independent boxes
 * overlap, and wslda_step replays every four steps as one captured CUDA
 * graph (one graph per history-slot phase and dt; per-kernel profiling falls
 * back to direct launches). Results are identical to direct execution. */
wslda_status wslda_set_graph(wslda_ctx* ctx, int enable, int nstreams);

/* Launch variant (cluster size, threads, lanes per pencil) the autotuner chose
 * for the box's stage kernels at wslda_start, as text. Setting the environment
 * variable WSLDA_VARIANT=<index> before creating a context forces a variant. */
wslda_status wslda_get_variant(wslda_ctx* ctx, int box, char* desc, int len);

/* Simulation time and steps taken (including start-up steps). */
wslda_status wslda_get_time(wslda_ctx* ctx, double* t, int64_t* steps);

/* Device bytes held by the context. */
int64_t wslda_memory_bytes(const wslda_ctx* ctx);

/* Uniform (plane-wave) BCS solution on the lattice k-set (Sec. 5.2.1, "inittype 0";
 * reduced 2x2 problem of Eq. HpsiEpsi). With u_k, v_k = (U_k, V_k) e^{ik.r}/sqrt(V),
 * xi_k = k^2/2 - mu_eff, E_k = sqrt(xi_k^2 + Delta^2) over all M lattice k:
 *  - the number equation (1/V) sum_k V_k^2 = rho_sigma fixes mu_eff = mu - U;
 *  - kind SLDA_A1: Delta = delta0 is given; 1/g_eff = -(1/V) sum_k 1/(2E_k)
 *    fixes C through Eq. Creg (C = rho^(1/3)/(1/g_eff + Lambda_c)), then
 *    U = B eF(rho) - Delta^2/(3 C rho^(2/3)) and mu = U + mu_eff;
 *  - kind BDG: the gap equation 1/(4 pi a) - Lambda_c = -(1/V) sum_k 1/(2E_k)
 *    is solved for Delta (first root on a log grid, 1e-6..8), U = 0, mu = mu_eff.
 * fn supplies kind, B, inv_4pi_a and ec (<= 0: zone-corner cutoff). */
typedef struct {
  double mu_eff, delta, mu, U, C, lam, inv_g;
} wslda_uniform;
wslda_status wslda_uniform_solve(const wslda_lattice* lat, const wslda_functional* fn, double rho_sigma,
                                 double delta0, wslda_uniform* out);

/* Fill a box with the positive-energy plane-wave states of a uniform solution
 * (mu_eff, delta > 0), computed on the device. State i takes the flattened
 * k index kidx[i] (host int64 [n]) or i when kidx is NULL (then n <= M).
 * Weights are set to T = 0. Replaces wslda_load_states. An aslda box (whole
 * spectrum) takes n/2 such states (n even; kidx then has n/2 entries) followed
 * by their negative-energy partners [v^*, -u^*], with the T = 0 weights of
 * both signs of E. */
wslda_status wslda_fill_uniform_states(wslda_ctx* ctx, int box, double mu_eff, double delta, const int64_t* kidx);

/* Replace the frozen weights (Sec. 2.5) of the loaded states, before
 * wslda_start: w_minus = f(-E_n), w_plus = f(E_n), host [n] doubles (NULL:
 * the T = 0 values 1 and 0). Non-finite weights give WSLDA_ENAN. */
wslda_status wslda_set_weights(wslda_ctx* ctx, int box, const double* w_minus, const double* w_plus);

/* Multiply component `comp` (0 = u, 1 = v) of every loaded state of the box
 * by a site-dependent complex factor phase[r] ([M] complex, host or device),
 * before wslda_start. With phase = e^{i theta(r)} on u this imprints the
 * phase theta on nu = sum u v^* and hence on Delta = -g_eff nu while leaving
 * rho and the normalisation unchanged: the vortex-line start of the
 * elongated-trap workload (theta the azimuthal angle about a line along z;
 * vortex dynamics is among the applications of Sec. 6). Factors of modulus
 * other than 1 are applied as given (the states are then not normalised).
 * The product is formed in double and rounded to the stored precision. */
wslda_status wslda_imprint_phase(wslda_ctx* ctx, int box, int comp, const double* phase, int on_device);

/* FP64 fused multiply-add throughput of the current CUDA device in TFLOP/s
 * (2 flops per FMA), the best of `reps` timed launches of a kernel of
 * independent FMA chains over every SM (CUDA events on the legacy default
 * stream, after one warm-up launch). A hardware microbenchmark, not part of
 * the method: it is the measured peak against which the FP64 step's
 * ALU-bound stage kernels are reported. Changes no device setting. */
wslda_status wslda_measure_fp64_rate(int reps, double* tflops);
/* FP64 addition throughput of the current device in tera-operations per
 * second (one addition per instruction), measured the same way: the ceiling
 * of FP64 work made of unfused additions and multiplications, such as the
 * butterflies of the transforms. A microbenchmark, not a step of the method. */
wslda_status wslda_measure_fp64_add_rate(int reps, double* tops);

/* Static self-consistent solve (Alg. 1, Sec. 3.2) of a trapped, spin-symmetric
 * T = 0 system, whose positive-energy eigenstates then become the box's states
 * (ready for wslda_start). Iteration i applies the map K of Alg. 1 to the
 * potentials p = (U, Delta): the matrix of Eq. HpsiEpsi built from p (Laplacian
 * of Eq. D2, W = U + V_ext - mu) is diagonalised, the densities of its M
 * positive-energy eigenstates give K[p] through the functional, with the
 * regulator Lambda_c of Eq. Creg evaluated at the input mean field; then
 * p <- m K[p] + (1 - m) p (linear mixing). The iteration stops when, from the
 * second iteration on, every energy term of Sec. 3.2 and the total change by
 * less than eps_energy * e_ref between consecutive iterations (Eq. E-conv) and,
 * with a particle-number target, |N_req - N_sigma| < eps_npart (Eq. N-conv);
 * with a target, Eq. update-mu is one more step of K and mu is mixed with the
 * potentials. method 1 replaces the linear mixing by modified Broyden mixing
 * (Sec. 3.2; D. D. Johnson, Phys. Rev. B 38, 12807 (1988), weights 1 and w_0,
 * the last broyden_memory iterations) of the vector (U, Delta, mu), with
 * alpha = mixing; its first iteration mixes linearly.
 *  - Requirements: the box holds nstates = M states; V_ext, U0 and delta0 are
 *    real and symmetric under the reflections i -> N - i (mod N) of every axis
 *    (a potential centred on site N/2); Delta_ext is zero. The problem is then
 *    real and splits into the 8 reflection-parity blocks, each diagonalised in
 *    double precision; otherwise WSLDA_EINVAL.
 *  - U0, delta0: initial potentials, host [M] doubles (Delta real).
 *  - qp_energies: host [M] output (nullable): the quasiparticle energy of each
 *    returned state, in state order.
 *  - On return the box's states are the eigenstates of the last matrix
 *    diagonalised (normalised, T = 0 weights) and its functional's mu is the
 *    final mu. The mixed path rounds the states to complex float.
 *  - out->iters, converged, mu, max_rel_change (last iteration's largest
 *    |change| / e_ref), n_sigma and the energy terms of the last iteration. */
typedef struct {
  double mixing;     /* m of the linear mixing, 0 < m <= 1 */
  double eps_energy; /* Eq. E-conv threshold */
  double e_ref;      /* energy scale of Eq. E-conv; <= 0: 1/2 (Fermi energy at k_F = 1) */
  int max_iters;     /* >= 1 */
  double n_target;   /* Eq. update-mu target N_sigma; <= 0: fixed mu */
  double a_mu;       /* Eq. update-mu step size */
  double eps_npart;  /* Eq. N-conv tolerance */
  int method;        /* 0 linear mixing, 1 modified Broyden mixing */
  int broyden_memory;   /* iterations kept, 1..8; <= 0: 7 */
  double broyden_w0;    /* regularisation weight w_0; <= 0: 0.01 */
  int fp32_iters;       /* leading iterations that diagonalise in single precision (a cheaper
                           approach to the fixed point); convergence is judged only between
                           two double-precision iterations; 0: double throughout */
} wslda_scf_params;
typedef struct {
  int iters, converged;
  double mu, max_rel_change, n_sigma;
  wslda_energy energy;
} wslda_scf_result;
wslda_status wslda_static_solve(wslda_ctx* ctx, int box, const double* U0, const double* delta0,
                                const wslda_scf_params* params, double* qp_energies, wslda_scf_result* out);

/* Densities rho [M] and nu [M complex] of device-resident states, without any
 * device allocation. The paper has no counterpart: this entry point exists for
 * callers that cannot call cudaMalloc, such as code whose device memory is all
 * owned by its own pool allocator, or code on a latency-critical path where
 * cudaMalloc (which can synchronise the device and can fail) is not acceptable.
 *  - uv: device pointer to [nstates][2][M] complex, float2 elements for
 *    WSLDA_MIXED and double2 for WSLDA_FP64; w_minus / w_plus: device [nstates]
 *    doubles or NULL (T = 0: 1 and 0); rho, nu: device outputs (nu interleaved).
 *  - Scratch is a fixed 16 MiB device array inside the library (every GPU that
 *    loads the library holds it until the process exits); lattices with more
 *    than 699050 sites (3 M > 2^21 doubles) are rejected with WSLDA_ENOMEM.
 *  - The first call on a device resolves that array's device address (a
 *    one-time set-up); make that first call before any stream capture. The
 *    address is kept for the life of the process: do not call this entry
 *    point after a cudaDeviceReset of that device.
 *  - The work is queued on `stream` (a cudaStream_t, NULL = default stream)
 *    and the call returns without waiting. All calls share the one scratch
 *    array, so calls that overlap on the GPU (other streams, other threads)
 *    race and give wrong results; serialise them. */
wslda_status wslda_densities_noalloc(int precision, const void* uv, const double* w_minus, const double* w_plus,
                                     int64_t nstates, int nx, int ny, int nz, double* rho, double* nu, void* stream);

/* Learned starting fields for the static solver (a companion of Alg. 1, not a
 * method of the paper): a network of four 3x3x3 convolutions with periodic
 * wrap-around, channels 2 -> hidden -> hidden -> hidden -> 2, tanh between
 * layers, mapping per-site (V_ext / eF, coupling) to (U / eF, Delta / eF).
 * Weights: float32 master copy, used rounded to bfloat16 (nearest even).
 * The convolutions run on the tensor cores as implicit GEMMs with bfloat16
 * operands and float32 accumulation: each layer's input (an activation, or
 * in the backward pass the gradient that the input-gradient convolution
 * consumes) is rounded to bfloat16 (nearest even) as it is staged; the
 * weight gradient uses the same rounded layer inputs. Activations, stored
 * gradients, the loss and Adam (b1 0.9, b2 0.999, eps 1e-8) are float32. Parameters are flattened per layer as W[co][ci][27] (offset
 * (dx, dy, dz) in {-1, 0, 1}^3 at (dx+1)*9 + (dy+1)*3 + (dz+1)) then bias[co];
 * a layer computes y[b][co][r] = bias[co] + sum_ci sum_d W[co][ci][d]
 * x[b][ci][r + d]. Activations are device float arrays [batch][2][M]; the
 * calls queue work on `stream` (a cudaStream_t); loss_grad synchronises it.
 *  - create: hidden is 8 or 32; up to max_batch samples per call; parameters
 *    start at zero (set them with set_params, host floats; this also resets
 *    Adam's moments).
 *  - loss_grad: forward, mean squared error against the targets, backward;
 *    the gradient stays in the network for adam() and is copied to grad_host
 *    when that pointer is not NULL.
 *  - symmetrize: average of each of nfields fields over the reflections
 *    i -> N - i (mod N) of the three axes (out must not alias y).
 *  - get_activation: the output of layer 0, 1 or 2 (after tanh, [batch][hidden]
 *    [M] floats) of the last forward or loss_grad call, copied to `out` (host
 *    or device memory); the call synchronises `stream`.
 *  - A tensor-core completion wait that gives up (bounded, about 2 s) makes
 *    loss_grad return WSLDA_ETIMEOUT. */
typedef struct wslda_net wslda_net;
wslda_status wslda_net_create(int nx, int ny, int nz, int hidden, int max_batch, wslda_net** out);
void wslda_net_destroy(wslda_net* net);
const char* wslda_net_last_error(const wslda_net* net);
int64_t wslda_net_param_count(const wslda_net* net);
wslda_status wslda_net_set_params(wslda_net* net, const float* theta);
wslda_status wslda_net_get_params(wslda_net* net, float* theta);
wslda_status wslda_net_forward(wslda_net* net, const float* x, int batch, float* y, void* stream);
wslda_status wslda_net_loss_grad(wslda_net* net, const float* x, const float* target, int batch, double* loss,
                                 float* grad_host, void* stream);
wslda_status wslda_net_adam(wslda_net* net, double lr, void* stream);
wslda_status wslda_net_symmetrize(const float* y, int64_t nfields, int nx, int ny, int nz, float* out, void* stream);
wslda_status wslda_net_get_activation(wslda_net* net, int layer, int batch, float* out, void* stream);

/* Per-kernel timing: when enabled, every launch is bracketed by CUDA events on
 * the context's stream and its duration is added to the kernel's total.
 * kind: 0 stage X (predictor), 1 stage Y (corrector), 2 density reduction
 * (with A != 1 also the per-stage current: derivative launch and sum over
 * states), 3 potentials, 4 start-up / diagnostics and, with A != 1, the
 * current-term launches that precede every application of H. */
wslda_status wslda_set_profiling(wslda_ctx* ctx, int enable);
wslda_status wslda_get_kernel_time(wslda_ctx* ctx, int kind, double* total_ms, int64_t* launches);

/* Number of kernels the context has launched so far (a graph replay counts
 * the kernels it contains). */
int64_t wslda_launch_count(const wslda_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* WSLDA_TD_H */
