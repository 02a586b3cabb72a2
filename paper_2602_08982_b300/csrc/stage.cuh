// Fused per-state kernels of the TDSLDA step.
//
// One thread-block cluster of CS CTAs owns one quasiparticle state (u, v).
// CTA `rank` keeps the x-slab [rank*P, (rank+1)*P) of both components in
// shared memory (P = NX / CS), rows padded to an odd pitch so that per-thread
// z-pencils are bank-conflict free. The kinetic term T phi = -1/2 lap phi is a
// 3D FFT (Eq. derivative-spectral, Nyquist kept) done as
//   z-forward, y-forward   (local pencils)
//   x-forward, * k^2/2, x-inverse   (pencils gathered across the cluster
//                                     through distributed shared memory)
//   y-inverse, z-inverse   (local)
// and the result stays on chip for the pointwise epilogue of the mode:
//   MODE_X   f(phi) = -i[H - <H>_n] phi (Eq. ABM-f), AB4 predictor and the
//            AM5 partial sum (Alg. 2 step 1), normalisation of the predictor
//            (Alg. 2 step 2). Reads phi, f_{k-2..k-4}; writes f_{k-1},
//            phi_p (over phi) and the partial sum c (over f_{k-4}).
//   MODE_Y   f(phi_p), corrector completion c + 251/720 dt f (Alg. 2 step 4),
//            normalisation (Alg. 2 step 8). Reads phi_p and c; writes phi.
//   MODE_F   f(phi) into a separate buffer (start-up history, diagnostics).
//   MODE_HORNER  out = base + coef [H - E_n] in (one Horner step of the
//            Taylor series of Eq. Taylor-exp); E_n = <in|H|in> is computed and
//            stored when requested, else read; optional normalisation.
//   MODE_EKIN    per-state <u|T|u>, <v|T|v> for the kinetic energy.
//   MODE_LAP     per-state contributions to the quantum-friction fields
//            (Sec. 5.2.4): w- Im(v lap v^*) - w+ Im(u lap u^*) (the divergence
//            of j by the product rule) and -(w- - w+)/2 (u lap v^* + v^* lap u)
//            (the sum in theta_B'), stored in h0 as [n][2][M] complex.
//   MODE_GRAD    the three Cartesian derivatives d_d of u and v (symbol
//            i k_d, Nyquist mode zeroed) and the per-state weighted
//            contributions to tau and j_d (Eqs. nab3D..jab3D), stored in h0.
//   MODE_AGRAD   the current term of h (Eq. h_sigma, A != 1) of the input
//            states: -i S with S = sum_d A_d d_d phi + (div A / 2) phi, stored
//            in h0, and the per-CTA partials of sum_r Re(phi^* (-i S)) (the
//            current part of <H>_n). The stage modes add it to H phi when
//            `cur` is set.
//   MODE_KALPHA  the part of the kinetic term of Eq. kinop-alpha that needs a
//            transform of the product alpha phi (spin-imbalanced ASLDA, alpha
//            varying in space): adds +1/2 T(alpha_a u) to the u row and
//            -1/2 T(alpha_b v) to the v row of h0 (which holds the current term
//            already), and adds Re sum_r [u^* T(alpha_a u) - v^* T(alpha_b v)]
//            (its whole kinetic part of <H>_n, T being Hermitian) to the per-CTA
//            partials in ecur. T = -1/2 lap with the Nyquist mode kept.
//   Both derivative modes use 1D transforms along one axis per derivative
//   (the symbol i k_d is diagonal in k_d, so the other two axes need no
//   transform): the slab is loaded once per axis (the second and third loads
//   come from L2), z and y locally, x across the cluster, each followed by a
//   pointwise sweep that accumulates into h0.
// Normalisation (Alg. 2 steps 2 and 8) is deferred: states are written as
// computed, each CTA stores its partial norm, a small kernel turns the partials
// into the per-state factor 1/sqrt(norm), and every consumer (the next stage,
// the density reduction, read-out) applies that factor on load. The only
// cluster barriers are the two around the x pass; CTAs exit without waiting. Per-state reductions (<H>_n, norms) are summed per thread in
// the working precision, then across threads and CTAs in double in a fixed
// order, so all CTAs of the cluster obtain bit-identical values.
#pragma once
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fft.cuh"

namespace wslda {
namespace cg = cooperative_groups;

template <typename R> struct fx4_of;
template <> struct fx4_of<float> { using type = float4; };
template <> struct fx4_of<double> { using type = double4; };
template <typename R> using fx4 = typename fx4_of<R>::type;

// MODE_X3 / MODE_X5: the predictor stage of AB3AM4 / AB5AM5 (MODE_X is AB4AM5's).
enum Mode : int {
  MODE_X = 0, MODE_Y = 1, MODE_F = 2, MODE_HORNER = 3, MODE_EKIN = 4, MODE_GRAD = 5, MODE_X3 = 6, MODE_X5 = 7,
  MODE_LAP = 8, MODE_AGRAD = 9, MODE_KALPHA = 10, NMODES = 11
};
// Modes that apply H (the only ones with a general-functional instance).
__host__ __device__ constexpr bool applies_h(int m) {
  return m == MODE_X || m == MODE_Y || m == MODE_F || m == MODE_HORNER || m == MODE_X3 || m == MODE_X5;
}

template <typename R>
struct StageArgs {
  cx<R>* phi;        // X, Y: phi slot; F, HORNER, EKIN: input states
  cx<R>* h0;         // X: receives f_{k-1};            F: output f;  HORNER: output
  const cx<R>* h1;   // X: f_{k-2}                                   HORNER: base
  const cx<R>* h2;   // X: f_{k-3}
  cx<R>* h3;         // X: f_{k-4} in, c out;  X5: f_{k-4};  Y: c in
  cx<R>* h4;         // X5: f_{k-5} in, c out (X3 reads f_{k-2}, f_{k-3} from h1, h2 and writes c over h2)
  const fx4<R>* WD;  // [M] {U + V_ext - mu, Re, Im (Delta + Delta_ext), 0}
  const R* ktab;     // [2 (NX+NY+NZ)]: per-slot k_d^2 * 0.5 / M, then k_d / M with the Nyquist mode zeroed
  const cx<R>* tw;   // [NX+NY+NZ] W_N^k per axis (used where a pencil spans lanes)
  double* E;         // HORNER: per-state shift (written when compute_e)
  double* out2;      // EKIN: [n][2] <u|T|u>, <v|T|v>
  const double* sc_in;    // [n] scale of the input states (true phi = sc_in * stored)
  const double* sc_base;  // HORNER: [n] scale of the base states
  double* sc_out;         // [n] scale of the written states: 1 for outputs that are not normalised
  double* npart;          // [n][16] per-CTA norm partials of normalised outputs (finalised by a separate kernel)
  int* err;          // error word: bit 0 non-finite norm
  double dt;
  double dV;
  double coef_re, coef_im;  // HORNER coefficient
  double ycoef;      // Y: coefficient of the new term of the corrector (251/720 for AM5, 9/24 for AM4)
  const double* wm;  // GRAD: frozen weights f(-E_n), f(E_n)
  const double* wp;
  const fx4<R>* av;  // AGRAD: [M] {A_x, A_y, A_z, div A / 2} (current potential, A != 1) of the u row
  const fx4<R>* av2; // AGRAD: the same for the v row (NULL: av; spin-imbalanced ASLDA: A_b)
  const cx<R>* alf;  // KALPHA and the general H modes: [M] {alpha_a / 2, alpha_b / 2} (NULL: constant A)
  const cx<R>* cur;  // X, Y, F, HORNER: current term -(i/2){A, grad} phi of the input states (NULL: none)
  double* ecur;      // AGRAD, KALPHA: write / add, stage modes read: [n][16] per-CTA partials of their <H>_n part
  int compute_e;
  int normalize;
  int nstates;
};

// Predictor-stage coefficients: b[j] multiplies f_{k-1-j} in the predictor
// (Eqs. AB3, AB4, AB5), a[j] in the corrector partial (Eqs. AM4, AM5 without
// the new term); D = history values read from memory (f_{k-1} is on chip).
template <int MODE> struct Scheme { static constexpr int D = 0; };
template <> struct Scheme<MODE_X3> {  // AB3AM4
  static constexpr int D = 2;
  static constexpr double b[5] = {23.0 / 12.0, -16.0 / 12.0, 5.0 / 12.0, 0.0, 0.0};
  static constexpr double a[4] = {19.0 / 24.0, -5.0 / 24.0, 1.0 / 24.0, 0.0};
};
template <> struct Scheme<MODE_X> {  // AB4AM5
  static constexpr int D = 3;
  static constexpr double b[5] = {55.0 / 24.0, -59.0 / 24.0, 37.0 / 24.0, -9.0 / 24.0, 0.0};
  static constexpr double a[4] = {646.0 / 720.0, -264.0 / 720.0, 106.0 / 720.0, -19.0 / 720.0};
};
template <> struct Scheme<MODE_X5> {  // AB5AM5
  static constexpr int D = 4;
  static constexpr double b[5] = {1901.0 / 720.0, -2774.0 / 720.0, 2616.0 / 720.0, -1274.0 / 720.0, 251.0 / 720.0};
  static constexpr double a[4] = {646.0 / 720.0, -264.0 / 720.0, 106.0 / 720.0, -19.0 / 720.0};
};

template <typename R_, int NX_, int NY_, int NZ_, int CS_, int BT_, int TX_, int TY_, int TZ_, int MINB_ = 1>
struct Geometry {
  using R = R_;
  using C = cx<R_>;
  static constexpr int NX = NX_, NY = NY_, NZ = NZ_, CS = CS_, BT = BT_;
  static constexpr int TX = TX_, TY = TY_, TZ = TZ_;
  static constexpr int MINB = MINB_;        // CTAs per SM the register budget is sized for
  // a budget of at most ~85 registers per thread (3 CTAs per SM, or 2 of 384+ threads)
  static constexpr bool TIGHT = MINB_ >= 3 || BT_ * MINB_ >= 768;
  // sites per thread per batch in the epilogues (fewer under a tight register budget)
  static constexpr int U = sizeof(R_) == 4 ? (TIGHT ? 2 : 4) : 2;
  static constexpr int P = NX / CS;         // x-planes per CTA
  // Row pitch TZ x (an odd number >= NZ / TZ): the TZ lanes of a z pencil read
  // consecutive elements and the rows of a warp start TZ elements apart modulo
  // the bank period, so a z pass touches each bank once per wavefront (TZ = 1:
  // an odd pitch; TZ = 4, NZ = 96: 100).
  static constexpr int ZP = TZ * ((NZ / TZ) % 2 == 0 ? NZ / TZ + 1 : NZ / TZ);
  static constexpr int SLAB = P * NY * ZP;  // complex elements per component
  static constexpr int NS = P * NY * NZ;    // sites per CTA
  static constexpr int M = NX * NY * NZ;
  static constexpr int NW = BT / 32;
  static constexpr int NCOL = 2 * NY * NZ / CS;  // x-pencils per CTA
  static constexpr size_t smem_bytes =
      size_t(2) * SLAB * sizeof(C) + size_t(NX + NY + NZ) * (2 * sizeof(R) + sizeof(C)) + 112 * sizeof(double) + 16;
  // reduction scratch (doubles): warp partials A [0,32) and B [32,64), per-CTA
  // slots of the <H>_n / kinetic sums [64, 96)
  static constexpr int RED_WA = 0, RED_WB = 32, RED_E = 64, RED_N = 96;
  static constexpr int RED_BAR = 104;  // 8-byte slot of the slab-load mbarrier
  // slab rows are 16-byte aligned in both memories: the slab arrives as one
  // bulk copy per row (TMA unit) on an mbarrier instead of per-element cp.async
  static constexpr bool BULK = (ZP * sizeof(C)) % 16 == 0 && (NZ * sizeof(C)) % 16 == 0;
  static_assert(NX % CS == 0, "cluster must split x evenly");
  static_assert((2 * NY * NZ) % CS == 0, "columns must split evenly");
  static_assert(BT % 32 == 0 && BT % TX == 0 && BT % TY == 0 && BT % TZ == 0, "block");
  static_assert(CS <= 16 && BT <= 1024, "cluster size / block size");
};

// Asynchronous global -> shared copies (8 or 16 bytes), all in flight at once.
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem_dst, const void* gmem_src) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
// Bulk L2 prefetch of a contiguous range (a hint: no completion to wait for).
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(p), "r"(bytes) : "memory");
}

// 32-bit shared::cluster addresses of this CTA's `p` in CTA `rank` of the cluster.
__device__ __forceinline__ unsigned dsmem_addr(const void* p, unsigned rank) {
  const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(p));
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ float2 ld_dsmem(unsigned addr, float2) {
  float2 v;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ double2 ld_dsmem(unsigned addr, double2) {
  double2 v;
  asm volatile("ld.shared::cluster.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(addr) : "memory");
  return v;
}
template <unsigned OFF>
__device__ __forceinline__ float2 ld_dsmem_off(unsigned addr, float2) {
  float2 v;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2+%3];" : "=f"(v.x), "=f"(v.y) : "r"(addr), "n"(OFF) : "memory");
  return v;
}
template <unsigned OFF>
__device__ __forceinline__ double2 ld_dsmem_off(unsigned addr, double2) {
  double2 v;
  asm volatile("ld.shared::cluster.v2.f64 {%0, %1}, [%2+%3];" : "=d"(v.x), "=d"(v.y) : "r"(addr), "n"(OFF) : "memory");
  return v;
}
template <unsigned OFF>
__device__ __forceinline__ void st_dsmem_off(unsigned addr, float2 v) {
  asm volatile("st.shared::cluster.v2.f32 [%0+%1], {%2, %3};" ::"r"(addr), "n"(OFF), "f"(v.x), "f"(v.y) : "memory");
}
template <unsigned OFF>
__device__ __forceinline__ void st_dsmem_off(unsigned addr, double2 v) {
  asm volatile("st.shared::cluster.v2.f64 [%0+%1], {%2, %3};" ::"r"(addr), "n"(OFF), "d"(v.x), "d"(v.y) : "memory");
}
__device__ __forceinline__ void st_dsmem(unsigned addr, float2 v) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ void st_dsmem(unsigned addr, double2 v) {
  asm volatile("st.shared::cluster.v2.f64 [%0], {%1, %2};" ::"r"(addr), "d"(v.x), "d"(v.y) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// mbarrier-completed bulk copies (global -> shared, one row each).
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void* src, unsigned bytes, unsigned bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}
// The same copy with an L2 eviction policy for the source lines.
__device__ __forceinline__ void bulk_g2s_hint(unsigned dst, const void* src, unsigned bytes, unsigned bar,
                                              uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
      ::"r"(dst), "l"(src), "r"(bytes), "r"(bar), "l"(pol) : "memory");
}

// L2 eviction priorities. The stages that apply H re-read their input state
// in the epilogue, tens of microseconds after the slab copy brought it in;
// meanwhile the history reads and the output writes stream several times
// that volume through L2. The slab copy marks the input lines evict-last, the
// epilogue's last read of them and every streaming access evict-first, so the
// re-read hits L2 instead of DRAM.
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ float2 ld_hint(const float2* p, uint64_t pol) {
  float2 v;
  asm volatile("ld.global.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ double2 ld_hint(const double2* p, uint64_t pol) {
  double2 v;
  asm volatile("ld.global.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;" : "=d"(v.x), "=d"(v.y) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ void st_hint(float2* p, float2 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(p), "f"(v.x), "f"(v.y), "l"(pol));
}
__device__ __forceinline__ void st_hint(double2* p, double2 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v2.f64 [%0], {%1, %2}, %3;" ::"l"(p), "d"(v.x), "d"(v.y), "l"(pol));
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned phase) {
  unsigned ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok) : "r"(bar), "r"(phase) : "memory");
  return ok != 0;
}
// Bounded wait for a phase of the barrier. Copies from valid global rows
// always complete; should the bound ever be reached, bit 2 of the error word
// is set (the host reports a timeout) and the wait continues, again bounded,
// so that no copy is left in flight into this CTA's shared memory on exit.
__device__ __forceinline__ void mbar_wait(unsigned bar, unsigned phase, int* err) {
  for (int round = 0; round < 2; ++round) {
    for (int it = 0; it < (1 << 22); ++it)
      if (mbar_try_wait(bar, phase)) return;
    if (err && round == 0 && threadIdx.x == 0) atomicOr(err, 4);
  }
}

// Local pencils along z (rows) or y, forward or inverse, over both components.
template <class G, int AXIS, bool INV>
__device__ __forceinline__ void local_pass(typename G::C* buf, const typename G::C* tw) {
  using C = typename G::C;
  constexpr int N = AXIS == 2 ? G::NZ : G::NY;
  constexpr int T = AXIS == 2 ? G::TZ : G::TY;
  constexpr int N1 = N / T;
  constexpr int NPEN = AXIS == 2 ? 2 * G::P * G::NY : 2 * G::P * G::NZ;
  constexpr int PER = G::BT / T;
  constexpr int ITERS = (NPEN + PER - 1) / PER;
  const int j = threadIdx.x % T;
#pragma unroll 1
  for (int it = 0; it < ITERS; ++it) {
    // a warp whose pencils all lie past the end has nothing to do (warp-uniform)
    if (it == ITERS - 1 && ITERS * PER > NPEN && (ITERS - 1) * PER + int(threadIdx.x & ~31u) / T >= NPEN) continue;
    const int p = it * PER + threadIdx.x / T;
    const bool act = p < NPEN;
    const int pp = act ? p : 0;
    C* base;
    int stride;
    if constexpr (AXIS == 2) {
      const int comp = pp / (G::P * G::NY), row = pp % (G::P * G::NY);
      base = buf + comp * G::SLAB + row * G::ZP;
      stride = 1;
    } else {
      const int comp = pp / (G::P * G::NZ), rem = pp % (G::P * G::NZ);
      const int xl = rem / G::NZ, z = rem % G::NZ;
      base = buf + comp * G::SLAB + xl * G::NY * G::ZP + z;
      stride = G::ZP;
    }
    C x[N1];
#pragma unroll
    for (int m = 0; m < N1; ++m) x[m] = base[(j + T * m) * stride];
    if constexpr (INV) pencil_inv<N, T>(x, j, tw);
    else pencil_fwd<N, T>(x, j, tw);
    if (act) {
#pragma unroll
      for (int m = 0; m < N1; ++m) base[(j + T * m) * stride] = x[m];
    }
  }
}

// Derivative along z (AXIS 2) or y (AXIS 1) by a 1D transform of the local
// pencils: forward, times i k_d / N_d (Nyquist mode zeroed), inverse.
template <class G, int AXIS>
__device__ __forceinline__ void local_deriv(typename G::C* buf, const typename G::R* ktab, const typename G::C* tw) {
  using C = typename G::C;
  using R = typename G::R;
  constexpr int N = AXIS == 2 ? G::NZ : G::NY;
  constexpr int T = AXIS == 2 ? G::TZ : G::TY;
  constexpr int N1 = N / T;
  constexpr int NPEN = AXIS == 2 ? 2 * G::P * G::NY : 2 * G::P * G::NZ;
  constexpr int PER = G::BT / T;
  constexpr int ITERS = (NPEN + PER - 1) / PER;
  // second half of ktab: k_d / M per slot; a 1D pass is normalised by 1/N
  constexpr int KOFF = G::NX + G::NY + G::NZ + G::NX + (AXIS == 2 ? G::NY : 0);
  const R fs = R(double(G::M) / double(N));
  const int j = threadIdx.x % T;
#pragma unroll 1
  for (int it = 0; it < ITERS; ++it) {
    // a warp whose pencils all lie past the end has nothing to do (warp-uniform)
    if (it == ITERS - 1 && ITERS * PER > NPEN && (ITERS - 1) * PER + int(threadIdx.x & ~31u) / T >= NPEN) continue;
    const int p = it * PER + threadIdx.x / T;
    const bool act = p < NPEN;
    const int pp = act ? p : 0;
    C* base;
    int stride;
    if constexpr (AXIS == 2) {
      const int comp = pp / (G::P * G::NY), row = pp % (G::P * G::NY);
      base = buf + comp * G::SLAB + row * G::ZP;
      stride = 1;
    } else {
      const int comp = pp / (G::P * G::NZ), rem = pp % (G::P * G::NZ);
      const int xl = rem / G::NZ, z = rem % G::NZ;
      base = buf + comp * G::SLAB + xl * G::NY * G::ZP + z;
      stride = G::ZP;
    }
    C x[N1];
#pragma unroll
    for (int m = 0; m < N1; ++m) x[m] = base[(j + T * m) * stride];
    pencil_fwd<N, T>(x, j, tw);
#pragma unroll
    for (int m = 0; m < N1; ++m) {
      const R kk = ktab[KOFF + j + T * m] * fs;
      x[m] = mk<C>(-kk * x[m].y, kk * x[m].x);
    }
    pencil_inv<N, T>(x, j, tw);
    if (act) {
#pragma unroll
      for (int m = 0; m < N1; ++m) base[(j + T * m) * stride] = x[m];
    }
  }
}

// x pencils across the cluster: forward, multiply by the kinetic symbol, inverse.
// Element x of a column lives in CTA x / P at plane x % P; the CTA windows are
// mapped once (mapa) and accessed with 32-bit ld/st.shared::cluster.
template <class G, bool GRAD = false>
__device__ __forceinline__ void x_pass(typename G::C* buf, const typename G::R* ktab, const typename G::C* tw,
                                       cg::cluster_group& cl, typename G::R& ekin_u, typename G::R& ekin_v,
                                       typename G::R gscale = 1) {
  using C = typename G::C;
  using R = typename G::R;
  constexpr int T = G::TX, N = G::NX, N1 = N / T;
  constexpr int PER = G::BT / T;
  constexpr int ITERS = (G::NCOL + PER - 1) / PER;
  constexpr unsigned PLANE = unsigned(G::NY * G::ZP * sizeof(C));
  const int j = threadIdx.x % T;
  const int rank = cl.block_rank();
  unsigned win[G::CS];
#pragma unroll
  for (int r = 0; r < G::CS; ++r) win[r] = dsmem_addr(buf, unsigned(r));
#pragma unroll 1
  for (int it = 0; it < ITERS; ++it) {
    // warp-uniform: no column left for this warp in the last round
    if (it == ITERS - 1 && ITERS * PER > G::NCOL && (ITERS - 1) * PER + int(threadIdx.x & ~31u) / T >= G::NCOL) continue;
    const int q = rank * G::NCOL + it * PER + threadIdx.x / T;
    const bool act = (it * PER + threadIdx.x / T) < G::NCOL;
    const int qq = act ? q : rank * G::NCOL;
    const int comp = qq / (G::NY * G::NZ), yz = qq % (G::NY * G::NZ);
    const int y = yz / G::NZ, z = yz % G::NZ;
    const unsigned off = unsigned((comp * G::SLAB + y * G::ZP + z) * sizeof(C));
    C x[N1];
    if constexpr (T == 1) {
      // one base address per CTA of the cluster, plane offsets as immediates
      unsigned base[G::CS];
#pragma unroll
      for (int r = 0; r < G::CS; ++r) base[r] = win[r] + off;
      static_for<0, N1>([&](auto mm) {
        constexpr int m = decltype(mm)::value;
        x[m] = ld_dsmem_off<unsigned(m % G::P) * PLANE>(base[m / G::P], C{});
      });
    } else {
#pragma unroll
      for (int m = 0; m < N1; ++m) {
        const int xg = j + T * m;
        x[m] = ld_dsmem(win[xg / G::P] + off + unsigned(xg % G::P) * PLANE, C{});
      }
    }
    pencil_fwd<N, T>(x, j, tw);
    if constexpr (GRAD) {
      // symbol i k_x (Nyquist mode zeroed): the second half of ktab holds
      // k_x / M, gscale turns it into the normalisation of the pass
      constexpr int K1 = G::NX + G::NY + G::NZ;
#pragma unroll
      for (int m = 0; m < N1; ++m) {
        const R kk = ktab[K1 + j + T * m] * gscale;
        x[m] = mk<C>(-kk * x[m].y, kk * x[m].x);
      }
    } else {
    const R kyz = ktab[G::NX + y] + ktab[G::NX + G::NY + z];
    // Parseval: sum_k (k^2/2M) |phi_k|^2 = <phi|T|phi> for the unnormalised FFT
    R ek = 0;
#pragma unroll
    for (int m = 0; m < N1; ++m) {
      const R kk = ktab[j + T * m] + kyz;
      ek += kk * (x[m].x * x[m].x + x[m].y * x[m].y);
      x[m] = scl(x[m], kk);
    }
    if (act) {
      if (comp == 0) ekin_u += ek;
      else ekin_v += ek;
    }
    }
    pencil_inv<N, T>(x, j, tw);
    // a column is read and written only by its own lane group: no barrier here
    if (act) {
      if constexpr (T == 1) {
        unsigned base[G::CS];
#pragma unroll
        for (int r = 0; r < G::CS; ++r) base[r] = win[r] + off;
        static_for<0, N1>([&](auto mm) {
          constexpr int m = decltype(mm)::value;
          st_dsmem_off<unsigned(m % G::P) * PLANE>(base[m / G::P], x[m]);
        });
      } else {
#pragma unroll
        for (int m = 0; m < N1; ++m) {
          const int xg = j + T * m;
          st_dsmem(win[xg / G::P] + off + unsigned(xg % G::P) * PLANE, x[m]);
        }
      }
    }
  }
}

// One state of a stage, inlined into the kernel (so that the arguments stay
// kernel parameters, read where they are used).
// GEN = false: the kinetic term is A T with a constant A folded into the
// symbol, one potential W for both rows, and no current term (A = 1, BdG).
// GEN = true adds, when the pointers are set, the current term `cur` and its
// <H>_n partials `ecur`; with `alf` (spin-imbalanced ASLDA) the rows take
// alpha_a/2 T u and -alpha_b/2 T v, the v row its own W_b (fourth field), and
// the kinetic part of <H>_n comes from the KALPHA partials instead of Parseval.
template <class G, int MODE, bool GEN>
__device__ __forceinline__ void stage_state(const StageArgs<typename G::R>& a, const int n, const int ncl,
                                            const unsigned iter = 0) {
  using C = typename G::C;
  using R = typename G::R;
  extern __shared__ __align__(16) unsigned char smem[];
  C* buf = reinterpret_cast<C*>(smem);
  R* ktab = reinterpret_cast<R*>(buf + 2 * G::SLAB);
  C* tws = reinterpret_cast<C*>(ktab + 2 * (G::NX + G::NY + G::NZ));
  double* red = reinterpret_cast<double*>(tws + (G::NX + G::NY + G::NZ));
  red = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(red) + 7) & ~uintptr_t(7));
  const fx4<R>* WD = a.WD;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = cl.block_rank();
  const int tid = threadIdx.x;
  const int gs0 = rank * G::NS;  // first global site of this slab
  constexpr int U = G::U;
  auto sidx = [](int s) { return (s / G::NZ) * G::ZP + (s % G::NZ); };
  const C* twx = tws;
  const C* twy = tws + G::NX;
  const C* twz = tws + G::NX + G::NY;
  const size_t sbase = size_t(n) * 2 * G::M;
  const C* in = a.phi + sbase;
  const unsigned bar = static_cast<unsigned>(__cvta_generic_to_shared(red + G::RED_BAR));
  // load the slab of both components (asynchronous copies, all in flight)
  if constexpr (G::BULK) {
    // one bulk copy per z row, issued by the first warp, completing on the barrier
    if (tid < 32) {
      if (tid == 0) mbar_arrive_expect_tx(bar, unsigned(2 * G::NS * sizeof(C)));
      __syncwarp();
      const unsigned b0 = static_cast<unsigned>(__cvta_generic_to_shared(buf));
      const uint64_t keep = policy_evict_last();
      for (int r = tid; r < 2 * G::P * G::NY; r += 32) {
        const int comp = r / (G::P * G::NY), row = r % (G::P * G::NY);
        const unsigned d = b0 + unsigned((comp * G::SLAB + row * G::ZP) * sizeof(C));
        const C* src = in + comp * G::M + gs0 + row * G::NZ;
        if constexpr (applies_h(MODE)) bulk_g2s_hint(d, src, unsigned(G::NZ * sizeof(C)), bar, keep);
        else bulk_g2s(d, src, unsigned(G::NZ * sizeof(C)), bar);
      }
    }
  } else {
    for (int i = tid; i < 2 * G::NS; i += G::BT) {
      const int comp = i / G::NS, s = i % G::NS;
      cp_async<sizeof(C)>(buf + comp * G::SLAB + sidx(s), in + comp * G::M + gs0 + s);
    }
  }
  // Prologue sweep over the slab: the potential part of <H>_n,
  // sum_r W (|u|^2 - |v|^2) + 2 Re(u^* D v), of the scaled input (the slab
  // itself stays unscaled; the FFT is linear, so the scale is applied to its
  // results instead). The first batch of a thread's field loads is issued
  // before the wait for the slab, so both round trips overlap.
  constexpr bool XM = MODE == MODE_X || MODE == MODE_X3 || MODE == MODE_X5;  // a predictor stage
  const bool need_e = XM || MODE == MODE_Y || MODE == MODE_F || (MODE == MODE_HORNER && a.compute_e);
  const bool spin2 = GEN && a.alf != nullptr;  // per-site alpha, W_b in the fourth field
  constexpr int UPMAX = G::TIGHT ? 4 : 16;  // fewer under a tight register budget
  constexpr int UP = (G::NS + G::BT - 1) / G::BT < UPMAX ? (G::NS + G::BT - 1) / G::BT : UPMAX;
  fx4<R> wd[UP];
  auto load_wd = [&](int s0) {
#pragma unroll
    for (int k = 0; k < UP; ++k) {
      const int s = s0 + k * G::BT;
      if (s < G::NS) wd[k] = WD[gs0 + s];
    }
  };
  if (need_e) load_wd(tid);
  if constexpr (MODE == MODE_Y) {
    // the corrector partial c (one state pass) starts moving into L2 with the slab
    if (tid < 2) prefetch_l2(a.h3 + sbase + size_t(tid) * G::M + gs0, unsigned(G::NS * sizeof(C)));
  }
  const R sin_ = R(a.sc_in[n]);
  if constexpr (G::BULK) mbar_wait(bar, iter & 1u, a.err);
  else cp_async_wait_all();
  __syncthreads();
  R ep = 0, ec = 0;  // compensated partial sum
  for (int s0 = tid; s0 < G::NS && need_e; s0 += G::BT * UP) {
    if (s0 != tid) load_wd(s0);
#pragma unroll
    for (int k = 0; k < UP; ++k) {
      const int s = s0 + k * G::BT;
      if (s < G::NS) {
        const C u = scl(buf[sidx(s)], sin_), v = scl(buf[G::SLAB + sidx(s)], sin_);
        const C dv = mul(mk<C>(wd[k].y, wd[k].z), v);
        const R wb = spin2 ? wd[k].w : wd[k].x;
        const R t = (wd[k].x * (u.x * u.x + u.y * u.y) - wb * (v.x * v.x + v.y * v.y) + R(2) * (u.x * dv.x + u.y * dv.y)) - ec;
        const R ns = ep + t;
        ec = (ns - ep) - t;
        ep = ns;
      }
    }
  }

  __syncthreads();  // the slab is read above before the z pass overwrites it
  if constexpr (MODE == MODE_KALPHA) {
    // the transform acts on alpha_a u and alpha_b v
    for (int s = tid; s < G::NS; s += G::BT) {
      const cx<R> al = a.alf[gs0 + s];
      buf[sidx(s)] = scl(buf[sidx(s)], R(2) * al.x);
      buf[G::SLAB + sidx(s)] = scl(buf[G::SLAB + sidx(s)], R(2) * al.y);
    }
    __syncthreads();
  }
  const R sin2 = sin_ * sin_;
  local_pass<G, 2, false>(buf, twz);
  __syncthreads();
  local_pass<G, 1, false>(buf, twy);
  cl.sync();
  // the next state's input slab starts moving into L2 while this one is transformed
  if (tid < 2 && n + ncl < a.nstates)
    prefetch_l2(a.phi + size_t(n + ncl) * 2 * G::M + size_t(tid) * G::M + gs0, unsigned(G::NS * sizeof(C)));
  R eku = 0, ekv = 0;
  x_pass<G>(buf, ktab, twx, cl, eku, ekv);
  // Publish this CTA's partial <H>_n (or kinetic sums) into the slots of every
  // CTA of the cluster on the barrier that closes the x pass; afterwards each
  // CTA reads only its own shared memory, so no CTA has to outlive another.
  double* slot = red + G::RED_E;
  {
    double v0 = MODE == MODE_EKIN ? double(eku)
                : (spin2 ? double(ep) : double(ep) + (double(eku) - double(ekv)) * double(sin2));
    double v1 = double(ekv);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      v0 += __shfl_xor_sync(0xffffffffu, v0, o);
      v1 += __shfl_xor_sync(0xffffffffu, v1, o);
    }
    if ((tid & 31) == 0) { red[G::RED_WA + (tid >> 5)] = v0; red[G::RED_WB + (tid >> 5)] = v1; }
    __syncthreads();
    if (tid < G::CS) {
      double s0 = 0.0, s1 = 0.0;
      for (int i = 0; i < G::NW; ++i) { s0 += red[G::RED_WA + i]; s1 += red[G::RED_WB + i]; }
      double* dst = cl.map_shared_rank(slot, tid);
      dst[rank] = s0;
      dst[G::CS + rank] = s1;
    }
  }
  cl.sync();
  // The epilogue's DRAM inputs (history slabs) start moving into L2 now, a
  // few microseconds before they are read.
  if (tid < 2) {
    const size_t off = sbase + size_t(tid) * G::M + gs0;
    constexpr unsigned nb = unsigned(G::NS * sizeof(C));
    if constexpr (XM) {
      prefetch_l2(a.h1 + off, nb);
      prefetch_l2(a.h2 + off, nb);
      if constexpr (Scheme<MODE>::D >= 3) prefetch_l2(a.h3 + off, nb);
      if constexpr (Scheme<MODE>::D >= 4) prefetch_l2(a.h4 + off, nb);
    }
  }
  double En = 0.0, Ev = 0.0;
  for (int r = 0; r < G::CS; ++r) { En += slot[r]; Ev += slot[G::CS + r]; }
  if constexpr (GEN)
    if (a.ecur)
      for (int r = 0; r < G::CS; ++r) En += a.ecur[size_t(n) * 16 + r];
  En *= a.dV;
  Ev *= a.dV;
  if (MODE == MODE_EKIN) { En *= double(sin2); Ev *= double(sin2); }
  local_pass<G, 1, true>(buf, twy);
  __syncthreads();
  local_pass<G, 2, true>(buf, twz);
  __syncthreads();
  // buf now holds T phi = -1/2 lap phi of this slab (natural order).

  if constexpr (MODE == MODE_EKIN) {
    if (rank == 0 && tid == 0) { a.out2[2 * n] = En; a.out2[2 * n + 1] = Ev; }
    return;
  } else if constexpr (MODE == MODE_LAP) {
    // buf holds T phi = -1/2 lap phi: lap = -2 T
    const R wmn = R(a.wm[n]), wpn = R(a.wp[n]), dw = wmn - wpn;
    C* out = a.h0 + sbase;
    for (int s = tid; s < G::NS; s += G::BT) {
      const int g = gs0 + s;
      const C uu = scl(in[g], sin_), vv = scl(in[G::M + g], sin_);
      const C lu = scl(buf[sidx(s)], R(-2) * sin_), lv = scl(buf[G::SLAB + sidx(s)], R(-2) * sin_);
      const C vlv = mulc(vv, lv), ulu = mulc(uu, lu);  // v conj(lap v), u conj(lap u)
      const R divj = wmn * vlv.y - wpn * ulu.y;
      const C bp = scl(add(mulc(uu, lv), mulc(lu, vv)), R(-0.5) * dw);  // u conj(lap v) + conj(v) lap u
      out[g] = mk<C>(divj, R(0));
      out[G::M + g] = bp;
    }
    return;
  } else if constexpr (MODE == MODE_KALPHA) {
    // buf holds T(alpha phi) of the stored (unscaled) slab
    C* out = a.h0 + sbase;
    R kp = 0, kc = 0;  // compensated partial of Re sum [u^* T(alpha_a u) - v^* T(alpha_b v)]
    for (int s = tid; s < G::NS; s += G::BT) {
      const int g = gs0 + s;
      const C uu = scl(in[g], sin_), vv = scl(in[G::M + g], sin_);
      const C tu = scl(buf[sidx(s)], sin_), tv = scl(buf[G::SLAB + sidx(s)], sin_);
      out[g] = add(out[g], scl(tu, R(0.5)));
      out[G::M + g] = sub(out[G::M + g], scl(tv, R(0.5)));
      const R t = (uu.x * tu.x + uu.y * tu.y - vv.x * tv.x - vv.y * tv.y) - kc;
      const R ns = kp + t;
      kc = (ns - kp) - t;
      kp = ns;
    }
    double v = double(kp);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) red[G::RED_WB + (tid >> 5)] = v;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int i = 0; i < G::NW; ++i) t += red[G::RED_WB + i];
      a.ecur[size_t(n) * 16 + rank] += t;  // the current-term launch wrote this CTA's slot
    }
    return;
  } else {
    if (MODE == MODE_HORNER) {
      if (a.compute_e) {
        if (rank == 0 && tid == 0) a.E[n] = En;
      } else {
        En = a.E[n];
      }
    }
    const R Er = R(En);
    R np = 0, nc = 0;  // compensated norm partial
    const bool norm_out = XM || MODE == MODE_Y || (MODE == MODE_HORNER && a.normalize);
    C* dst = (MODE == MODE_HORNER || MODE == MODE_F) ? a.h0 + sbase : a.phi + sbase;
    const R dt = R(a.dt);
    const R sbase_ = MODE == MODE_HORNER ? R(a.sc_base[n]) : R(1);
    // one pointwise sweep: H phi on the fly, f = -i (H - <H>_n) phi, integrator;
    // results go straight to global memory (normalisation deferred)
    constexpr int D = Scheme<MODE>::D;
    // sites per batch: fewer with five history reads; the corrector and the
    // other single-input modes keep 4 in flight even under a tight budget
    // (their epilogue holds far fewer values per site)
    constexpr int UE = XM ? ((D >= 4 && U > 2) ? U / 2 : U) : (sizeof(R) == 4 ? 4 : U);
    const uint64_t pf = policy_evict_first();
    for (int s0 = tid; s0 < G::NS; s0 += G::BT * UE) {
      C u[UE], v[UE], x1[2][UE], x2[2][UE], x3[2][UE], x4[2][D >= 4 ? UE : 1];
      fx4<R> wd[UE];
#pragma unroll
      for (int k = 0; k < UE; ++k) {
        const int s = s0 + k * G::BT;
        if (s < G::NS) {
          const int g = gs0 + s;
          u[k] = ld_hint(in + g, pf);
          v[k] = ld_hint(in + G::M + g, pf);
          wd[k] = WD[g];
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const size_t gg = sbase + c * G::M + g;
            if constexpr (XM) {
              x1[c][k] = ld_hint(a.h1 + gg, pf);
              x2[c][k] = ld_hint(a.h2 + gg, pf);
              if constexpr (D >= 3) x3[c][k] = ld_hint(a.h3 + gg, pf);
              if constexpr (D >= 4) x4[c][k] = ld_hint(a.h4 + gg, pf);
            }
            if constexpr (MODE == MODE_Y) x3[c][k] = ld_hint(a.h3 + gg, pf);
            if constexpr (MODE == MODE_HORNER) x1[c][k] = a.h1[gg];
          }
        }
      }
#pragma unroll
      for (int k = 0; k < UE; ++k) {
        const int s = s0 + k * G::BT;
        if (s < G::NS) {
          const int g = gs0 + s;
          const int b = sidx(s);
          const C uu = scl(u[k], sin_), vv = scl(v[k], sin_);
          const R w = wd[k].x;
          const C d = mk<C>(wd[k].y, wd[k].z);
          // (H - <H>_n) phi for both components (Eq. dpsidt-Hpsi; A T phi from the symbol)
          R ka = sin_, kb = sin_, wb = w;
          if constexpr (GEN) {
            if (spin2) {  // Eq. kinop-alpha: alpha/2 T on each row, W_b on the v row
              const cx<R> al = a.alf[g];
              ka *= al.x;
              kb *= al.y;
              wb = wd[k].w;
            }
          }
          C hm[2];
          hm[0] = sub(add(add(scl(buf[b], ka), scl(uu, w)), mul(d, vv)), scl(uu, Er));
          hm[1] = sub(sub(sub(mulc(uu, d), scl(buf[G::SLAB + b], kb)), scl(vv, wb)), scl(vv, Er));
          if constexpr (GEN) {
            if (a.cur) {  // current term (and with alf the transformed alpha phi parts)
              hm[0] = add(hm[0], a.cur[sbase + g]);
              hm[1] = add(hm[1], a.cur[sbase + G::M + g]);
            }
          }
          const C ph[2] = {uu, vv};
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const size_t gg = sbase + c * G::M + g;
            C res;
            if constexpr (XM) {
              using S = Scheme<MODE>;
              const C fv = mul_mi(hm[c]);  // f(phi) = -i (H - <H>_n) phi
              // predictor phi + dt sum_j b_j f_{k-1-j}, corrector partial phi + dt sum_j a_j f_{k-1-j}
              C pb = add(scl(fv, R(S::b[0])), scl(x1[c][k], R(S::b[1])));
              C pa = add(scl(fv, R(S::a[0])), scl(x1[c][k], R(S::a[1])));
              pb = add(pb, scl(x2[c][k], R(S::b[2])));
              pa = add(pa, scl(x2[c][k], R(S::a[2])));
              if constexpr (D >= 3) {
                pb = add(pb, scl(x3[c][k], R(S::b[3])));
                pa = add(pa, scl(x3[c][k], R(S::a[3])));
              }
              if constexpr (D >= 4) pb = add(pb, scl(x4[c][k], R(S::b[4])));
              res = add(ph[c], scl(pb, dt));
              const C corr = add(ph[c], scl(pa, dt));
              st_hint(a.h0 + gg, fv, pf);
              if constexpr (D == 2) st_hint(const_cast<C*>(a.h2) + gg, corr, pf);  // over f_{k-3}, its last use
              if constexpr (D == 3) st_hint(a.h3 + gg, corr, pf);                  // over f_{k-4}
              if constexpr (D == 4) st_hint(a.h4 + gg, corr, pf);                  // over f_{k-5}
            } else if constexpr (MODE == MODE_Y) {
              res = add(x3[c][k], scl(mul_mi(hm[c]), R(a.ycoef * a.dt)));
            } else if constexpr (MODE == MODE_F) {
              res = mul_mi(hm[c]);
            } else {  // HORNER: out = base + coef (H - E) in
              res = add(scl(x1[c][k], sbase_), mul(mk<C>(R(a.coef_re), R(a.coef_im)), hm[c]));
            }
            st_hint(dst + c * G::M + g, res, pf);
            if (norm_out) {
              const R t = (res.x * res.x + res.y * res.y) - nc;
              const R ns = np + t;
              nc = (ns - np) - t;
              np = ns;
            }
          }
        }
      }
    }
    // Norm partials go to global memory (finalised into 1/sqrt(norm) by a
    // separate kernel); outputs that are not normalised get the factor 1.
    if (norm_out) {
      double v = double(np);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if ((tid & 31) == 0) red[G::RED_WB + (tid >> 5)] = v;
      __syncthreads();
      if (tid == 0) {
        double t = 0.0;
        for (int i = 0; i < G::NW; ++i) t += red[G::RED_WB + i];
        a.npart[size_t(n) * 16 + rank] = t;
      }
    } else if (rank == 0 && tid == 0 && a.sc_out) {
      a.sc_out[n] = 1.0;
    }
  }
}

// MODE_GRAD / MODE_AGRAD for one state: derivatives along z, y, x in turn,
// each from a fresh load of the input slab, each followed by its sweep.
template <class G, int MODE>
__device__ __forceinline__ void deriv_state(const StageArgs<typename G::R>& a, const int n, const int ncl,
                                            const unsigned iter = 0) {
  using C = typename G::C;
  using R = typename G::R;
  extern __shared__ __align__(16) unsigned char smem[];
  C* buf = reinterpret_cast<C*>(smem);
  R* ktab = reinterpret_cast<R*>(buf + 2 * G::SLAB);
  C* tws = reinterpret_cast<C*>(ktab + 2 * (G::NX + G::NY + G::NZ));
  double* red = reinterpret_cast<double*>(tws + (G::NX + G::NY + G::NZ));
  red = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(red) + 7) & ~uintptr_t(7));
  cg::cluster_group cl = cg::this_cluster();
  const int rank = cl.block_rank();
  const int tid = threadIdx.x;
  const int gs0 = rank * G::NS;
  auto sidx = [](int s) { return (s / G::NZ) * G::ZP + (s % G::NZ); };
  const size_t sbase = size_t(n) * 2 * G::M;
  const C* in = a.phi + sbase;
  C* out = a.h0 + sbase;
  const R sin_ = R(a.sc_in[n]);
  R wmn = 0, wpn = 0;
  if constexpr (MODE == MODE_GRAD) {
    wmn = R(a.wm[n]);
    wpn = R(a.wp[n]);
  }
  if (tid < 2 && n + ncl < a.nstates)
    prefetch_l2(a.phi + size_t(n + ncl) * 2 * G::M + size_t(tid) * G::M + gs0, unsigned(G::NS * sizeof(C)));
  R ep = 0, ec = 0;  // AGRAD: compensated partial of sum Re(phi^* G)
  const unsigned bar = static_cast<unsigned>(__cvta_generic_to_shared(red + G::RED_BAR));
#pragma unroll 1
  for (int d = 2; d >= 0; --d) {
    if (d != 2) __syncthreads();  // the previous sweep has read the slab
    if constexpr (G::BULK) {
      // one bulk copy per z row on the slab barrier: completion 3 iter + (2 - d)
      if (tid < 32) {
        if (tid == 0) mbar_arrive_expect_tx(bar, unsigned(2 * G::NS * sizeof(C)));
        __syncwarp();
        const unsigned b0 = static_cast<unsigned>(__cvta_generic_to_shared(buf));
        for (int r = tid; r < 2 * G::P * G::NY; r += 32) {
          const int comp = r / (G::P * G::NY), row = r % (G::P * G::NY);
          bulk_g2s(b0 + unsigned((comp * G::SLAB + row * G::ZP) * sizeof(C)), in + comp * G::M + gs0 + row * G::NZ,
                   unsigned(G::NZ * sizeof(C)), bar);
        }
      }
      mbar_wait(bar, (3u * iter + unsigned(2 - d)) & 1u, a.err);
    } else {
      for (int i = tid; i < 2 * G::NS; i += G::BT) {
        const int comp = i / G::NS, s = i % G::NS;
        cp_async<sizeof(C)>(buf + comp * G::SLAB + sidx(s), in + comp * G::M + gs0 + s);
      }
      cp_async_wait_all();
    }
    __syncthreads();
    if (d == 2) {
      local_deriv<G, 2>(buf, ktab, tws + G::NX + G::NY);
    } else if (d == 1) {
      local_deriv<G, 1>(buf, ktab, tws + G::NX);
    } else {
      cl.sync();  // every CTA holds its fresh slab and has finished its y sweep
      R e0 = 0, e1 = 0;
      x_pass<G, true>(buf, ktab, tws, cl, e0, e1, R(double(G::M) / double(G::NX)));
      cl.sync();  // every column is back in place
    }
    __syncthreads();
    for (int s = tid; s < G::NS; s += G::BT) {
      const int g = gs0 + s;
      const C du = scl(buf[sidx(s)], sin_), dv = scl(buf[G::SLAB + sidx(s)], sin_);
      const C uu = scl(in[g], sin_), vv = scl(in[G::M + g], sin_);
      if constexpr (MODE == MODE_GRAD) {
        // tau_d = w-|d v|^2 + w+|d u|^2, j_d = w- Im(v d v^*) - w+ Im(u d u^*),
        // stored as {tau, j_x}, {j_y, j_z}, tau summed over the directions
        const R tau = wmn * (dv.x * dv.x + dv.y * dv.y) + wpn * (du.x * du.x + du.y * du.y);
        const R jd = wmn * (vv.y * dv.x - vv.x * dv.y) - wpn * (uu.y * du.x - uu.x * du.y);
        if (d == 2) {
          out[g] = mk<C>(tau, R(0));
          out[G::M + g] = mk<C>(R(0), jd);
        } else if (d == 1) {
          C o0 = out[g];
          o0.x += tau;
          out[g] = o0;
          C o1 = out[G::M + g];
          o1.x = jd;
          out[G::M + g] = o1;
        } else {
          C o0 = out[g];
          o0.x += tau;
          o0.y = jd;
          out[g] = o0;
        }
      } else {
        const fx4<R> av = a.av[g];
        const fx4<R> bv = a.av2 ? a.av2[g] : av;  // the v row's current potential
        const R Ad = d == 0 ? av.x : (d == 1 ? av.y : av.z);
        const R Bd = d == 0 ? bv.x : (d == 1 ? bv.y : bv.z);
        C su, sv;
        if (d == 2) {
          su = scl(uu, av.w);
          sv = scl(vv, bv.w);
        } else {
          su = out[g];
          sv = out[G::M + g];
        }
        su = add(su, scl(du, Ad));
        sv = add(sv, scl(dv, Bd));
        if (d == 0) {
          su = mul_mi(su);
          sv = mul_mi(sv);
          const R t = (uu.x * su.x + uu.y * su.y + vv.x * sv.x + vv.y * sv.y) - ec;
          const R ns = ep + t;
          ec = (ns - ep) - t;
          ep = ns;
        }
        out[g] = su;
        out[G::M + g] = sv;
      }
    }
  }
  if constexpr (MODE == MODE_AGRAD) {
    double v = double(ep);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) red[G::RED_WB + (tid >> 5)] = v;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int i = 0; i < G::NW; ++i) t += red[G::RED_WB + i];
      a.ecur[size_t(n) * 16 + rank] = t;
    }
  }
}

// PERSIST = false: one cluster per state. PERSIST = true: a cluster handles
// states n, n + ncl, ... (ncl clusters resident at once), prefetching the next
// state's input slab into L2 during the current one. Between states the whole
// CTA passes a barrier before the slab is overwritten; remote CTAs touch this
// slab and the reduction slots only after the next state's first cluster
// barrier. (The one-state form is a separate instance because the loop makes
// the compiler keep per-state invariants in registers.)
template <class G, int MODE, bool PERSIST, bool GEN = false>
__global__ void __launch_bounds__(G::BT, G::MINB) stage_kernel(const __grid_constant__ StageArgs<typename G::R> a) {
  using C = typename G::C;
  using R = typename G::R;
  extern __shared__ __align__(16) unsigned char smem[];
  C* buf = reinterpret_cast<C*>(smem);
  R* ktab = reinterpret_cast<R*>(buf + 2 * G::SLAB);
  C* tws = reinterpret_cast<C*>(ktab + 2 * (G::NX + G::NY + G::NZ));
  constexpr int NAX = G::NX + G::NY + G::NZ;
  for (int i = threadIdx.x; i < NAX; i += G::BT) {
    ktab[i] = a.ktab[i];
    ktab[NAX + i] = a.ktab[NAX + i];
    tws[i] = a.tw[i];
  }
  const int ncl = gridDim.x / G::CS;
  if constexpr (G::BULK) {
    if (threadIdx.x == 0) {
      double* red = reinterpret_cast<double*>(tws + NAX);
      red = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(red) + 7) & ~uintptr_t(7));
      mbar_init(static_cast<unsigned>(__cvta_generic_to_shared(red + G::RED_BAR)), 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
  }
  if constexpr (PERSIST) {
    unsigned iter = 0;
#pragma unroll 1
    for (int n = blockIdx.x / G::CS; n < a.nstates; n += ncl, ++iter) {
      __syncthreads();
      if constexpr (MODE == MODE_GRAD || MODE == MODE_AGRAD) deriv_state<G, MODE>(a, n, ncl, iter);
      else stage_state<G, MODE, GEN>(a, n, ncl, iter);
    }
  } else {
    __syncthreads();
    if constexpr (MODE == MODE_GRAD || MODE == MODE_AGRAD) deriv_state<G, MODE>(a, blockIdx.x / G::CS, ncl);
    else stage_state<G, MODE, GEN>(a, blockIdx.x / G::CS, ncl);
  }
}

}  // namespace wslda
