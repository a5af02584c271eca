// Device-side definitions shared by the AT-DNS kernels (sm_103a).
//
// Geometry of the periodic (2 pi)^3 grid cut into virtual PEs (Sec. 3,
// Eqs. (NT)-(NB)), the 4th- and 6th-order stencil coefficients (zero-delay
// rows of Table B, Appendix B), the Table B AT time weights and the
// Philox4x32-10 generator that stands in for the network delays of
// Algorithm 1.
#pragma once
#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

namespace atdns {

constexpr int kNumQ = 16;        // per-point derived fields: u, v, w, T, 12 fluxes
constexpr int kNumGhostQ = 9;    // per ghost point: 5 fluxes of the direction, u, v, w, T
constexpr int kNumGrad = 12;     // du_i/dx_j (i-major) then dT/dx_j
constexpr int kNumStat = 15;     // summed statistics per block
constexpr int kMaxModes = 128;   // forcing modes of the half set for kf <= 4
constexpr int kMaxKf = 4;

// Indices of the summed statistics.
enum StatIdx {
  ST_RHO = 0, ST_M0, ST_M1, ST_M2, ST_E, ST_KE, ST_SIGS, ST_G2, ST_G3, ST_G4,
  ST_ENST, ST_PTHETA, ST_FPOW, ST_U2, ST_C
};

// Health bits.
enum HealthBits { H_NONFINITE = 1, H_RHO = 2, H_P = 4 };

struct Geom {
  int n[3];          // points per direction
  int pes[3];        // PEs per direction
  int nl[3];         // points per PE per direction
  int xstate;        // what Table B's weights extrapolate at a delayed stencil
                     // point: 0 each differentiated quantity, 1 the state U
  long long npts;    // n0 n1 n2
  long long plane[3];// points of a plane normal to d: npts / n[d]
  long long stride[3];  // linear-index stride of direction d: 1, n0, n0 n1
  int M;             // stencil half width: 2 (4th order) or 3 (6th order)
  int nlev;          // ring levels L + T_l, T_l = M + 1
  // central stencil coefficients with the denominators and dx folded in
  double c1[3], c2[3], c3[3];         // D1 = sum_m c_m (f[+m] - f[-m])
  double a0[3], a1[3], a2[3], a3[3];  // D2 = a0 f + sum_m a_m (f[+m] + f[-m])
  double hloc[3];    // 1/(12 dx) (M = 2) or 1/(60 dx) (M = 3): one-sided stencils
  double inv_dx[3];  // 1/dx
};

// Central stencils of half width M = 2 (4th order, /12) or 3 (6th order:
// D1 (-1, 9, -45, 0, 45, -9, 1)/60, D2 (2, -27, 270, -490, 270, -27, 2)/180).
inline void set_stencils(Geom& g, int M) {
  g.M = M;
  for (int d = 0; d < 3; ++d) {
    const double dx = 2.0 * M_PI / g.n[d];
    if (M == 2) {
      g.c1[d] = 8.0 / (12.0 * dx);
      g.c2[d] = -1.0 / (12.0 * dx);
      g.c3[d] = 0.0;
      g.a0[d] = -30.0 / (12.0 * dx * dx);
      g.a1[d] = 16.0 / (12.0 * dx * dx);
      g.a2[d] = -1.0 / (12.0 * dx * dx);
      g.a3[d] = 0.0;
      g.hloc[d] = 1.0 / (12.0 * dx);
    } else {
      g.c1[d] = 45.0 / (60.0 * dx);
      g.c2[d] = -9.0 / (60.0 * dx);
      g.c3[d] = 1.0 / (60.0 * dx);
      g.a0[d] = -490.0 / (180.0 * dx * dx);
      g.a1[d] = 270.0 / (180.0 * dx * dx);
      g.a2[d] = -27.0 / (180.0 * dx * dx);
      g.a3[d] = 2.0 / (180.0 * dx * dx);
      g.hloc[d] = 1.0 / (60.0 * dx);
    }
    g.inv_dx[d] = 1.0 / dx;
  }
}

struct Phys {
  double gamma, gm1, prandtl, mu0, omega, cp_over_pr;
  int eform;         // 0: fifth variable E (total energy); 1: rho e (Eq. (ie))
  int vlaw;          // 0: mu0 T^omega; 1: Sutherland mu0 T^(3/2) (1 + S) / (T + S)
  double suth_s;     // S (Sutherland temperature over the reference temperature)
};

// Stencil coefficients and physical constants in the kernel's scalar type,
// converted once on the host (a conversion from double on the device would
// run on the FP64 pipe).
template <typename S>
struct Coef {
  S c1[3], c2[3], c3[3];          // D1 = sum_m c_m (f[+m] - f[-m])
  S a0[3], a1[3], a2[3], a3[3];   // D2 = a0 f + sum_m a_m (f[+m] + f[-m])
  S hloc[3];                      // scale of the one-sided stencils
  S gamma, gm1, mu0, omega, cp_over_pr;
  S inv_gamma;
  S dt;
  int eform, vlaw;                // energy form and viscosity law (Phys)
  S suth_s, suth_c;               // Sutherland S and mu0 (1 + S)
  // power law with omega = p/q (q <= 64): g = T^(omega - 1) is the root of
  // g^q T^(q - p) = 1 (vq = q, va = q - p); vrat = 0 when omega is no such
  // fraction
  int vrat, vq, va;
  float vexpm1;                   // omega - 1 (FP32 start value)
  S vinvq, vc2, mu0omega;         // 1/q, (q + 1)/(2 q^2), mu0 omega
};

template <typename S>
inline Coef<S> make_coef(const Geom& g, const Phys& ph, double dt) {
  Coef<S> c;
  for (int d = 0; d < 3; ++d) {
    c.c1[d] = (S)g.c1[d];
    c.c2[d] = (S)g.c2[d];
    c.c3[d] = (S)g.c3[d];
    c.a0[d] = (S)g.a0[d];
    c.a1[d] = (S)g.a1[d];
    c.a2[d] = (S)g.a2[d];
    c.a3[d] = (S)g.a3[d];
    c.hloc[d] = (S)g.hloc[d];
  }
  c.gamma = (S)ph.gamma;
  c.gm1 = (S)ph.gm1;
  c.mu0 = (S)ph.mu0;
  c.omega = (S)ph.omega;
  c.cp_over_pr = (S)ph.cp_over_pr;
  c.inv_gamma = (S)(1.0 / ph.gamma);
  c.dt = (S)dt;
  c.eform = ph.eform;
  c.vlaw = ph.vlaw;
  c.suth_s = (S)ph.suth_s;
  c.suth_c = (S)(ph.mu0 * (1.0 + ph.suth_s));
  c.vrat = 0;
  c.vq = 1;
  c.va = 0;
  for (int q = 1; q <= 64 && !ph.vlaw; ++q) {
    const double pq = ph.omega * q, pr = std::nearbyint(pq);
    if (std::fabs(pq - pr) <= 2e-15 * q && pr >= 0.0 && pr <= q) {
      c.vrat = 1;
      c.vq = q;
      c.va = q - (int)pr;
      break;
    }
  }
  c.vexpm1 = (float)(ph.omega - 1.0);
  c.vinvq = (S)(1.0 / c.vq);
  c.vc2 = (S)((c.vq + 1.0) / (2.0 * c.vq * c.vq));
  c.mu0omega = (S)(ph.mu0 * ph.omega);
  return c;
}

// Stencil coefficients and constants duplicated into both lanes of a pair
// (converted on the host, read from the parameter space).
struct CoefPair {
  float2 c1[3], c2[3];        // D1 = c1 (f[+1] - f[-1]) + c2 (f[+2] - f[-2])
  float2 nc1[3], nc2[3];      // -c1, -c2 (flux divergence)
  float2 a1[3], a2[3];        // D2 = a0 f + a1 (f[+1] + f[-1]) + a2 (f[+2] + f[-2])
  float2 a0[3], a0sum;        // a0 per direction, and their sum (Laplacian)
  float2 hloc[3];             // scale of the PE-local stencils (1 / (12 dx))
  float2 gamma, gm1, inv_gamma, cp_over_pr, mu0, mu0omega, dt;
};

inline CoefPair make_coef_pair(const Coef<float>& K) {
  CoefPair P;
  auto d2 = [](float a) { return make_float2(a, a); };
  for (int d = 0; d < 3; ++d) {
    P.c1[d] = d2(K.c1[d]);
    P.c2[d] = d2(K.c2[d]);
    P.nc1[d] = d2(-K.c1[d]);
    P.nc2[d] = d2(-K.c2[d]);
    P.a1[d] = d2(K.a1[d]);
    P.a2[d] = d2(K.a2[d]);
    P.a0[d] = d2(K.a0[d]);
    P.hloc[d] = d2(K.hloc[d]);
  }
  P.a0sum = d2(K.a0[0] + K.a0[1] + K.a0[2]);
  P.gamma = d2(K.gamma);
  P.gm1 = d2(K.gm1);
  P.inv_gamma = d2(K.inv_gamma);
  P.cp_over_pr = d2(K.cp_over_pr);
  P.mu0 = d2(K.mu0);
  P.mu0omega = d2(K.mu0omega);
  P.dt = d2(K.dt);
  return P;
}

// Sign/zero test on the bit pattern (no floating-point instruction).
__device__ __forceinline__ bool nonpositive(double v) { return __double_as_longlong(v) <= 0; }
__device__ __forceinline__ bool nonpositive(float v) { return __float_as_int(v) <= 0; }

// Linear index -> (x, y, z).  Grids hold fewer than 2^31 points (the create
// call checks), so 32-bit unsigned division suffices (a 64-bit integer
// division is a long software sequence).
__device__ __forceinline__ void decode(const Geom& g, long long idx, int& x, int& y, int& z) {
  const unsigned i = (unsigned)idx;
  const unsigned t = i / (unsigned)g.n[0];
  x = (int)(i - t * (unsigned)g.n[0]);
  z = (int)(t / (unsigned)g.n[1]);
  y = (int)(t - (unsigned)z * (unsigned)g.n[1]);
}

// Index of the point within the plane normal to d.
__device__ __forceinline__ long long plane_index(const Geom& g, int d, int x, int y, int z) {
  if (d == 0) return (long long)z * g.n[1] + y;
  if (d == 1) return (long long)z * g.n[0] + x;
  return (long long)y * g.n[0] + x;
}

// Ring slot of level m (m >= 0): m mod nlev, in 32 bits while the step count
// fits (a uniform branch; the 64-bit remainder is a long instruction sequence).
__device__ __forceinline__ int ring_slot(const Geom& g, long long m) {
  return m < 0x7fffffffLL ? (int)((unsigned)m % (unsigned)g.nlev) : (int)(m % g.nlev);
}

__device__ __forceinline__ int pe_number(const Geom& g, int x, int y, int z) {
  return ((z / g.nl[2]) * g.pes[1] + (y / g.nl[1])) * g.pes[0] + (x / g.nl[0]);
}

// Table B weights of levels n-k .. n-k-M (T_l = M + 1 levels), integers for
// integer k.  4th order: (k^2+3k+2)/2, -(k^2+2k), (k^2+k)/2.  6th order:
// (k^3+6k^2+11k+6)/6, -(k^3+5k^2+6k)/2, (k^3+4k^2+3k)/2, -(k^3+3k^2+2k)/6.
template <int M>
__device__ __forceinline__ void at_weights(int k, int (&w)[M + 1]) {
  if constexpr (M == 2) {
    w[0] = ((k + 1) * (k + 2)) / 2;
    w[1] = -(k * (k + 2));
    w[2] = (k * (k + 1)) / 2;
  } else {
    w[0] = ((k + 1) * (k + 2) * (k + 3)) / 6;
    w[1] = -((k * (k + 2) * (k + 3)) / 2);
    w[2] = (k * (k + 1) * (k + 3)) / 2;
    w[3] = -((k * (k + 1) * (k + 2)) / 6);
  }
}

// Philox4x32-10 (Salmon et al., SC'11): counter c, key k, ten rounds, key
// bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

constexpr uint32_t kDelayTag = 0x4154u;
constexpr uint32_t kForceTag = 0x464Fu;

// The random delay draw of face f of PE p at step n: uniform on {0..L} from
// word 0 of the counter-based generator.
__device__ __forceinline__ int delay_draw(long long n, int p, int f, int L, uint32_t k0, uint32_t k1) {
  const uint4 w = philox4x32_10(make_uint4((uint32_t)n, (uint32_t)p, (uint32_t)f, kDelayTag), k0, k1);
  return (int)(((unsigned long long)w.x * (unsigned long long)(L + 1)) >> 32);
}

// Delay of face f of PE p at step n (Sec. 3.1, Algorithms 1 and 2); the
// first L + T_l steps are synchronous.  Mode 4 (ordered random delays): the
// neighbour's messages arrive in order, so the newest level received ages by
// at most one step per step, k_n = min(d_n, k_{n-1} + 1) over the draws d of
// mode 2 with k = 0 before the start-up ends; unrolled, the minimum over
// j <= min(L, n - n0) of d_{n-j} + j and of n - n0 + 1 (a pure function of
// the step, like every other mode).
__device__ __forceinline__ int delay_of(int mode, long long n, int p, int f, int L, int tl, int cr,
                                        uint32_t k0, uint32_t k1) {
  const long long n0 = L + tl;
  if (mode == 0 || n < n0) return 0;
  if (mode == 1) return (int)((n - n0) % cr);
  if (mode == 3) return L;                  // fixed worst case (stability scans, Sec. 3.2)
  int k = delay_draw(n, p, f, L, k0, k1);
  if (mode == 4) {
    const long long jmax = n - n0 < L ? n - n0 : L;
    for (long long j = 1; j <= jmax; ++j) {
      const int c = delay_draw(n - j, p, f, L, k0, k1) + (int)j;
      k = c < k ? c : k;
    }
    if (n - n0 + 1 < k) k = (int)(n - n0 + 1);
  }
  return k;
}

// PE-local 4th-order first-derivative stencils of the mixed-derivative rule
// (Sec. 2.1), as (offset, coefficient x 12) rows indexed by kind: 0 central
// (1, -8, 0, 8, -1), 1 first point (-25, 48, -36, 16, -3) on 0..4, 2 second
// point (-3, -10, 18, -6, 1) on -1..3, 3 and 4 their mirror images at the last
// two points of a PE.  Central rows pad with a zero coefficient.
__constant__ int kLocalOff[5][5] = {
    {-2, -1, 1, 2, 0}, {0, 1, 2, 3, 4}, {-1, 0, 1, 2, 3}, {1, 0, -1, -2, -3}, {0, -1, -2, -3, -4}};
__constant__ float kLocalCoefF[5][5] = {
    {1, -8, 8, -1, 0}, {-25, 48, -36, 16, -3}, {-3, -10, 18, -6, 1}, {3, 10, -18, 6, -1}, {25, -48, 36, -16, 3}};
__constant__ double kLocalCoefD[5][5] = {
    {1, -8, 8, -1, 0}, {-25, 48, -36, 16, -3}, {-3, -10, 18, -6, 1}, {3, 10, -18, 6, -1}, {25, -48, 36, -16, 3}};
__device__ __forceinline__ float local_coef(float, int kind, int i) { return kLocalCoefF[kind][i]; }
__device__ __forceinline__ double local_coef(double, int kind, int i) { return kLocalCoefD[kind][i]; }

// The 6th-order set (coefficient x 60): 0 central (-1, 9, -45, 45, -9, 1);
// 1, 2, 3 the first three points of a PE on offsets 0..6, -1..5, -2..4;
// 4, 5, 6 the last three (mirror images of 3, 2, 1).
__constant__ int kLocal6Off[7][7] = {
    {-3, -2, -1, 1, 2, 3, 0},     {0, 1, 2, 3, 4, 5, 6},         {-1, 0, 1, 2, 3, 4, 5},
    {-2, -1, 0, 1, 2, 3, 4},      {2, 1, 0, -1, -2, -3, -4},     {1, 0, -1, -2, -3, -4, -5},
    {0, -1, -2, -3, -4, -5, -6}};
__constant__ double kLocal6Coef[7][7] = {
    {-1, 9, -45, 45, -9, 1, 0},           {-147, 360, -450, 400, -225, 72, -10},
    {-10, -77, 150, -100, 50, -15, 2},    {2, -24, -35, 80, -30, 8, -1},
    {-2, 24, 35, -80, 30, -8, 1},         {10, 77, -150, 100, -50, 15, -2},
    {147, -360, 450, -400, 225, -72, 10}};
__constant__ float kLocal6CoefF[7][7] = {
    {-1, 9, -45, 45, -9, 1, 0},           {-147, 360, -450, 400, -225, 72, -10},
    {-10, -77, 150, -100, 50, -15, 2},    {2, -24, -35, 80, -30, 8, -1},
    {-2, 24, 35, -80, 30, -8, 1},         {10, 77, -150, 100, -50, 15, -2},
    {147, -360, 450, -400, 225, -72, 10}};

// Row i of the PE-local stencil of `kind` for half width M: offset and
// coefficient (times the stencil denominator); 2M + 1 entries.
template <int M>
__device__ __forceinline__ int local_off(int kind, int i) {
  if constexpr (M == 2) return kLocalOff[kind][i];
  else return kLocal6Off[kind][i];
}
template <int M>
__device__ __forceinline__ float local_coefm(float, int kind, int i) {
  if constexpr (M == 2) return kLocalCoefF[kind][i];
  else return kLocal6CoefF[kind][i];
}
template <int M>
__device__ __forceinline__ double local_coefm(double, int kind, int i) {
  if constexpr (M == 2) return kLocalCoefD[kind][i];
  else return kLocal6Coef[kind][i];
}

// Order-preserving map of a double to a signed 64-bit key (for atomic min/max).
__device__ __forceinline__ long long ordered_key(double v) {
  long long b = __double_as_longlong(v);
  return b ^ ((b >> 63) & 0x7FFFFFFFFFFFFFFFLL);
}

__device__ __forceinline__ bool nonfinite(double v) {
  return ((unsigned long long)__double_as_longlong(v) & 0x7FF0000000000000ULL) == 0x7FF0000000000000ULL;
}
__device__ __forceinline__ bool nonfinite(float v) {
  return ((unsigned)__float_as_uint(v) & 0x7F800000u) == 0x7F800000u;
}

template <typename S> struct Vec2;
template <> struct Vec2<double> { using type = double2; };
template <> struct Vec2<float> { using type = float2; };
template <typename S> using vec2_t = typename Vec2<S>::type;

// Step state kept on the device, so that one captured step can be replayed:
// level n of the state, the forward-Euler flag of the first AB2 step and which
// of the two state buffers holds U^n.
struct DevState {
  long long n;
  int first;
  int cur;
  unsigned long long check;   // bounds-checked builds: index checks that failed (CheckBits)
};

// Bounds-checked builds (every translation unit compiled with -DAT_DNS_CHECKS):
// an index outside [0, n) is recorded in the device step state (the class of
// access as a CheckBits bit) and replaced by 0, so the access stays inside the
// buffer and the host reports the failure after the call (AT_DNS_E_BOUNDS).
// Ordinary builds return the index unchanged and compile no check.
enum CheckBits { CHK_STATE = 1, CHK_RING = 2, CHK_GHOST = 4, CHK_STAGE = 8 };
#ifdef AT_DNS_CHECKS
__device__ __forceinline__ long long checked(long long i, long long n, const DevState* ds, unsigned what) {
  if (i >= 0 && i < n) return i;
  if (ds) atomicOr(const_cast<unsigned long long*>(&ds->check), (unsigned long long)what);
  return 0;
}
#else
__device__ __forceinline__ long long checked(long long i, long long, const DevState*, unsigned) { return i; }
#endif

template <typename S>
struct StepArgs {
  const S* Ub[2];      // both state buffers; U^n is Ub[cur]
  S* Ulob[2];          // both low-word buffers (compensated form) or null
  const DevState* ds;  // device step state (null: U, Unext, ... below are used as given)
  const S* U;          // [5][npts] level n
  S* Unext;            // [5][npts] level n+1 (step) -- may be null for rhs-only
  const S* PQ;         // [16][npts]
  const S* G;          // [12][npts]
  const S* GH[3];      // [9][2M P_d][plane_d] per direction
  S* Rprev;            // [5][npts] R^{n-1} in, R^n out
  const S* Ulo;        // compensated form: low words of U (else null)
  S* Ulo_next;         // compensated form: low words of U^{n+1}
  double* Rout;        // rhs-only output [5][npts] or null
  S* xst;              // FP32 forms: U^{n+1} at the x-face slabs [hi, lo][5][2M P_x][plane_x] (else null)
  long long xst_half;  // elements from the hi half of xst to the lo half (0: no lo half)
  double* partial;     // [gridDim.x][kNumStat]
  unsigned long long* words;  // [0] max wave key, [1] min rho key, [2] min p key, [3] health
  const vec2_t<S>* fB; // forcing lines [(K+1)][3][n2][n1] or null
  const vec2_t<S>* fX; // exp(i kx x) table [(K+1)][n0]
  int fK;              // max |kx| of the forcing modes
  long long n;         // step of U
  double dt;
  int first;           // 1: forward Euler (no R^{n-1})
  int do_update;       // 1: write Unext/Rprev/ring; 0: write Rout
  int do_stats;
  int rk;              // 1: a stage of the low-storage RK3 (Rprev holds the stage register dU)
  S rkA, rkB;          // its coefficients: dU = rkA dU + dt R, U = U + rkB dU
};

// The per-step fields of one evaluation: from the device step state when the
// arguments carry one, else as given.  Kept apart from StepArgs so that the
// kernels read the (large) argument block from the parameter space and hold
// only these few values in registers.
template <typename S>
struct StepDyn {
  const S* U;          // [5][npts] level n
  S* Unext;            // [5][npts] level n+1
  const S* Ulo;        // compensated form: low words of U^n (else null)
  S* Ulo_next;         // compensated form: low words of U^{n+1}
  long long n;         // step of U
  int first;           // 1: forward Euler
};

template <typename S>
__device__ __forceinline__ StepDyn<S> resolve_step(const StepArgs<S>& A) {
  StepDyn<S> D;
  if (!A.ds) {
    D.U = A.U;
    D.Unext = A.Unext;
    D.Ulo = A.Ulo;
    D.Ulo_next = A.Ulo_next;
    D.n = A.n;
    D.first = A.first;
    return D;
  }
  const int cur = A.ds->cur;
  D.U = A.Ub[cur];
  D.Unext = const_cast<S*>(A.Ub[1 - cur]);
  D.Ulo = A.Ulob[cur];
  D.Ulo_next = A.Ulob[1 - cur];
  D.n = A.ds->n;
  D.first = A.ds->first;
  return D;
}

// Pressure from the conserved variables of one point: (gamma-1)(E - rho|u|^2/2)
// in the total-energy form, (gamma-1) rho e in the internal-energy form.
// The multiply-adds are explicit, so every kernel that inlines this gets the
// same rounding (an implicit contraction may differ between call sites).
template <typename S>
__device__ __forceinline__ S pressure(const Coef<S>& K, S m0, S m1, S m2, S u, S v, S w, S E) {
  return K.eform ? K.gm1 * E : K.gm1 * fma(S(-0.5), fma(m0, u, fma(m1, v, m2 * w)), E);
}

// Viscosity and its temperature derivative (Sec. 2): power law mu0 T^omega,
// or Sutherland mu0 T^(3/2) (1 + S) / (T + S).
// x^e for a small non-negative integer e (uniform over the grid), by squaring.
template <typename S>
__device__ __forceinline__ S ipow(S x, int e) {
  S r = S(1);
  while (e) {
    if (e & 1) r *= x;
    e >>= 1;
    if (e) x *= x;
  }
  return r;
}

// FP32 forms, power law: g = T^(omega - 1) by the hardware base-2 logarithm
// and exponential (a few ulp for the temperatures of a flow); mu = mu0 T g,
// dmu/dT = mu0 omega g
__device__ __forceinline__ void viscosity_power32(const Coef<float>& K, float T, float& mu, float& dmudT) {
  const float gg = __powf(T, K.vexpm1);
  mu = K.mu0 * T * gg;
  dmudT = K.mu0omega * gg;
}

template <typename S>
__device__ __forceinline__ void viscosity(const Coef<S>& K, S T, S& mu, S& dmudT) {
  if (K.vlaw) {
    const S inv = S(1) / (T + K.suth_s);
    mu = K.suth_c * T * sqrt(T) * inv;
    dmudT = mu * (S(1.5) / T - inv);
  } else if constexpr (sizeof(S) == 4) {
    viscosity_power32(K, T, mu, dmudT);
  } else if (K.vrat && T > S(1e-3) && T < S(1e3)) {
    // omega = p/q: g = T^(omega - 1) from an FP32 start g0, corrected as
    // g = g0 r^(-1/q) with r = g0^q T^(q - p) = 1 + d, taking two terms of the
    // binomial series (1 + d)^(-1/q) = 1 - d/q + (q + 1)/(2 q^2) d^2 - ...
    // (|d| < 1e-4, so the next term is below FP64 rounding).  Then
    // mu = mu0 T g and dmu/dT = mu0 omega g, with no division and no FP64
    // logarithm or exponential.
    const S g0 = (S)powf((float)T, K.vexpm1);
    const S d = ipow(g0, K.vq) * ipow(T, K.va) - S(1);
    const S gg = g0 * fma(d, fma(d, K.vc2, -K.vinvq), S(1));
    mu = K.mu0 * T * gg;
    dmudT = K.mu0omega * gg;
  } else {
    mu = K.mu0 * exp(K.omega * log(T));   // mu0 T^omega
    dmudT = K.omega * mu / T;
  }
}

// |x| by clearing the sign bit (integer instructions only).
__device__ __forceinline__ double abs_bits(double x) {
  return __longlong_as_double(__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFLL);
}
__device__ __forceinline__ float abs_bits(float x) { return __int_as_float(__float_as_int(x) & 0x7FFFFFFF); }

// 1/x rounded to nearest (the correctly rounded reciprocal instruction
// sequence for FP32, plain division for FP64).
__device__ __forceinline__ float rcp_rn(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp_rn(double x) { return 1.0 / x; }

// Separately rounded products / sums (never contracted into an FMA), for the
// error-free transformations of the compensated update.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }

// ---------------------------------------------------------------------------
// FP64 values in the FP32 forms with integer instructions only.  The slab ring
// of past levels is FP64 in every form; an FP64 (or FP32 <-> FP64 conversion)
// instruction in an FP32 kernel would run on the FP64 pipe, a few per cent of
// the FP32 rate on GB300, and a lane that takes it holds the whole warp.

// f as a double (exact for normal floats; subnormals flush to signed zero).
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xFFu;
  const unsigned long long sg = (unsigned long long)(b & 0x80000000u) << 32;
  if (e == 0u) return __longlong_as_double((long long)sg);
  const unsigned long long ed = e == 0xFFu ? 0x7FFULL : (unsigned long long)(e + 896u);
  return __longlong_as_double((long long)(sg | (ed << 52) | ((unsigned long long)(b & 0x7FFFFFu) << 29)));
}

// hi + lo as a double, for a renormalised pair (|lo| <= ulp(hi)/2, as the
// compensated update leaves it): hi's 24-bit significand widened to 53 bits
// plus lo's, aligned to it (lo's bits beyond the 53rd are truncated, a
// relative error below 2^-52).  Any other pair takes the FP64 add.
__device__ __forceinline__ double pair_to_double(float hi, float lo) {
  const unsigned bh = __float_as_uint(hi), bl = __float_as_uint(lo);
  const int eh = (int)((bh >> 23) & 0xFFu), el = (int)((bl >> 23) & 0xFFu);
  if (el == 0) return f2d_bits(hi);                        // lo is zero (or subnormal)
  if (eh == 0 || eh == 0xFF || el == 0xFF) return __dadd_rn(f2d_bits(hi), f2d_bits(lo));
  // hi = Mh 2^(eh-150) = M u with M = Mh 2^29, u = 2^(eh-179); lo = Ml 2^(el-eh+29) u
  const int sh = el - eh + 29;
  if (sh > 5) return __dadd_rn(f2d_bits(hi), f2d_bits(lo));
  unsigned long long M = (unsigned long long)((bh & 0x7FFFFFu) | 0x800000u) << 29;
  const unsigned long long Ml = (bl & 0x7FFFFFu) | 0x800000u;
  const unsigned long long add = sh >= 0 ? Ml << sh : (sh > -40 ? Ml >> (-sh) : 0ULL);
  int ed = eh + 896;
  if ((bh ^ bl) & 0x80000000u) {
    M -= add;                                               // >= 2^52 - 2^28
    if (M < (1ULL << 52)) { M <<= 1; ed -= 1; }
  } else {
    M += add;                                               // < 2^53 for a renormalised pair
  }
  return __longlong_as_double((long long)(((unsigned long long)(bh & 0x80000000u) << 32) |
                                          ((unsigned long long)ed << 52) | (M & 0xFFFFFFFFFFFFFULL)));
}

// d = hi + lo with hi = d truncated to 24 significant bits (exact) and lo the
// remaining 29 bits rounded to a float.  |d| below 2^-126 flushes to a signed
// zero; |d| of 2^128 or more, infinities and NaNs give an infinite or NaN hi.
__device__ __forceinline__ void split_double(double d, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned bh = (unsigned)(b >> 32), bl = (unsigned)b;
  const unsigned sg = bh & 0x80000000u;
  const int ef = (int)((bh >> 20) & 0x7FFu) - 896;           // biased float exponent
  lo = 0.f;
  if (ef <= 0) { hi = __uint_as_float(sg); return; }
  const unsigned mant = ((bh & 0xFFFFFu) << 3) | (bl >> 29);
  if (ef >= 255) {
    const bool nan = ((bh >> 20) & 0x7FFu) == 0x7FFu && ((bh & 0xFFFFFu) | bl) != 0u;
    hi = __uint_as_float(sg | 0x7F800000u | (nan ? 0x400000u : 0u));
    return;
  }
  hi = __uint_as_float(sg | ((unsigned)ef << 23) | mant);
  const unsigned r = bl & 0x1FFFFFFFu;                       // d - hi = +-r 2^(ef-179)
  const int es = ef - 52;                                    // biased exponent of 2^(ef-179)
  if (r != 0u && es > 0) lo = __uint_as_float(__float_as_uint((float)r * __uint_as_float((unsigned)es << 23)) | sg);
}

// x-face slabs of U^{n+1} staged in FP32 by the step kernels (FP32 forms): the
// next step's ghost kernel reads them, in the ring's slab layout, for its
// x-face work instead of strided loads of the state.  li: local x index of the
// point in its PE (nl points), pe: its PE in x, pl = z n1 + y; un / unlo: the
// new state and its low words.
template <typename S>
__device__ __forceinline__ void stage_xface(const Geom& g, const StepArgs<S>& A, int li, int pe, long long pl,
                                            const S (&un)[5], const S (&unlo)[5]) {
  const int M = g.M, nl = g.nl[0];
  if (!A.xst || g.pes[0] == 1 || (li >= M && li < nl - M)) return;
  const int t = li < M ? li : li - nl + 2 * M;
  const long long P2 = 2LL * M * g.pes[0];
  S* o = A.xst + (2LL * M * pe + t) * g.plane[0] + pl;
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    o[v * P2 * g.plane[0]] = un[v];
    if (A.xst_half) o[A.xst_half + v * P2 * g.plane[0]] = unlo[v];
  }
}

// The FP64 ring value of a state variable: the double itself, or hi + lo of
// the compensated FP32 form (lo = 0 in the plain FP32 form).
__device__ __forceinline__ double ring_value(double hi, double) { return hi; }
__device__ __forceinline__ double ring_value(float hi, float lo) { return pair_to_double(hi, lo); }

// AB2 update of the five variables of one point (Eq. (time_ab)):
// U^{n+1} = U^n + dt (3/2 R^n - 1/2 R^{n-1}), forward Euler on the first step.
// With low words (compensated FP32 form) the state is carried as hi + lo and
// the increment is added by TwoSum (Knuth), so no increment is lost below the
// resolution of the high word; the stencils read the high word only.
// Rp: R^{n-1} (or the RK3 stage register) of the point already loaded
// (null: read here).  A low-storage RK3 stage (A.rk) updates the register
// dU = rkA dU + dt R (kept in the Rprev array) and adds rkB dU to the state.
template <typename S>
__device__ __forceinline__ bool needs_rprev(const StepArgs<S>& A, const StepDyn<S>& D) {
  return A.do_update && (A.rk ? A.rkA != S(0) : !D.first);
}

// F: 0 AB2 step, 1 RK3 stage, 2 either (A.rk read per point).
// unlo: the low words of U^{n+1} (zero without compensation), for the ring.
// Lp: the low words of U^n of the point already loaded (null: read here).
template <int F, typename S>
__device__ __forceinline__ void ab2_update_v(const Coef<S>& K, const StepArgs<S>& A, const StepDyn<S>& D, long long idx,
                                             long long N, const S (&Uo)[5], const S (&R)[5], S (&un)[5],
                                             S (&unlo)[5], unsigned& health, const S* Rp, const S* Lp) {
  const bool ld = needs_rprev(A, D);
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    const S rp = ld ? (Rp ? Rp[v] : A.Rprev[v * N + idx]) : S(0);
    S inc, kept, scale;
    if (F == 2 ? A.rk != 0 : F == 1) {
      kept = fma(A.rkA, rp, K.dt * R[v]);   // stage register dU
      inc = A.rkB * kept;                   // the state grows by rkB dU
      scale = S(1);
    } else {
      inc = D.first ? R[v] : fma(S(1.5), R[v], S(-0.5) * rp);
      kept = R[v];
      scale = K.dt;
    }
    if (D.Ulo) {
      const S dlt = mul_rn(scale, inc);
      const S s = add_rn(Uo[v], dlt);                           // TwoSum(U_hi, dlt)
      const S bp = sub_rn(s, Uo[v]);
      const S e = add_rn(sub_rn(Uo[v], sub_rn(s, bp)), sub_rn(dlt, bp));
      const S lo = add_rn(Lp ? Lp[v] : D.Ulo[v * N + idx], e);
      const S hi = add_rn(s, lo);                               // renormalise
      unlo[v] = sub_rn(lo, sub_rn(hi, s));
      D.Ulo_next[v * N + idx] = unlo[v];
      un[v] = hi;
    } else {
      un[v] = fma(scale, inc, Uo[v]);
      unlo[v] = S(0);
    }
    D.Unext[v * N + idx] = un[v];
    A.Rprev[v * N + idx] = kept;
    if (nonfinite(un[v])) health |= H_NONFINITE;
  }
}

// In FP64 the RK3 and AB2 forms are separate code paths under one uniform
// branch, so that an AB2 step does not also issue the stage arithmetic on the
// FP64 pipe (the bound of the FP64 kernels); in FP32 one path for both keeps
// the register count down.
template <typename S>
__device__ __forceinline__ void ab2_update(const Coef<S>& K, const StepArgs<S>& A, const StepDyn<S>& D, long long idx,
                                           long long N, const S (&Uo)[5], const S (&R)[5], S (&un)[5],
                                           S (&unlo)[5], unsigned& health, const S* Rp = nullptr,
                                           const S* Lp = nullptr) {
  if constexpr (sizeof(S) == 8) {
    if (A.rk) ab2_update_v<1>(K, A, D, idx, N, Uo, R, un, unlo, health, Rp, Lp);
    else ab2_update_v<0>(K, A, D, idx, N, Uo, R, un, unlo, health, Rp, Lp);
  } else {
    ab2_update_v<2>(K, A, D, idx, N, Uo, R, un, unlo, health, Rp, Lp);
  }
}

}  // namespace atdns
