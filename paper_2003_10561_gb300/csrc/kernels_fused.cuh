// Fused AT-DNS step kernel: one pass over U per step.
//
// A CTA owns a TX x TY tile of one PE in x and y and marches in z through a
// chunk of ZC planes of one PE.  A shared-memory window holds, on the tile
// plus a two-cell halo in x and y, u, v, w for nine planes (z-4 .. z+4), and
// T, rho and H -- the quantity whose product with u_d is the fifth flux
// (E + p, or rho e) -- for seven (z-2 .. z+4): each field for as many planes
// as its stencils reach.  Halo cells beyond a PE face hold the
// AT ghost values of that direction (Table B extrapolation done by k_ghost),
// planes beyond a PE z-face hold the z ghosts, so every stencil of Sec. 2.1 is
// a plain read of the window:
//   * first / second derivatives of u, v, w, T in x, y, z;
//   * inviscid fluxes: each plane's x and y fluxes are formed once into shared
//     arrays (from the window, or from the ghost arrays across a PE face); the
//     column's z fluxes at z-2 .. z+2 are formed from the window (or the z
//     ghost arrays) at each plane, which keeps 25 registers free that a queue
//     carried across planes would hold;
//   * mixed derivatives: the central cross stencil D_a(D_b f) inside, and at
//     PE-boundary points the average of the PE-local derivative in a of the AT
//     derivative in b and vice versa.  The AT derivatives that the x- and
//     y-stencils take are formed once per plane into shared arrays (on
//     x-extended rows and y-extended columns, like the fluxes), so every lane
//     runs the same five-tap stencil of its own kind; the z-stencils take the
//     inner derivatives from the window (the one-sided reach of 4 planes in z
//     is why u, v, w are kept for nine planes).
// Then the assembly, forcing, AB2 (or RK3 stage) update, ring write and
// statistics of k_main.
// No per-point work arrays (derived fields, gradients) exist on this path.
//
// The tile shape is a template parameter so that every window access is one
// shared-memory load at a constant offset from one of nine per-plane bases.
#pragma once
#include "kernels.cuh"

namespace atdns {

constexpr int kWinPlanes = 9;   // u, v, w: planes z-4 .. z+4
constexpr int kWinT = 7;        // T: planes z-2 .. z+4
constexpr int kWinR = 7;        // rho, H: planes z-2 .. z+4
enum WinField { WF_U = 0, WF_V, WF_W, WF_T, WF_R, WF_H };
// per-plane AT derivatives for the mixed rule: on x-extended rows (taken by
// the x-stencils) and on y-extended columns (taken by the y-stencils)
enum XRField { XR_VY = 0, XR_WZ, XR_UY, XR_UZ };
enum YCField { YC_VX = 0, YC_UX, YC_WZ, YC_VZ };

template <int TX, int TY>
struct TileShape {
  static constexpr int CX = TX + 4, CY = TY + 4, CELLS = CX * CY;
  static constexpr int THREADS = TX * TY;
  // element offsets of the shared-memory regions
  static constexpr int OFF_A = 0;                                   // [9][3][CELLS]
  static constexpr int OFF_T = OFF_A + kWinPlanes * 3 * CELLS;      // [7][CELLS]
  static constexpr int OFF_R = OFF_T + kWinT * CELLS;               // [7][2][CELLS]
  static constexpr int OFF_FX = OFF_R + kWinR * 2 * CELLS;          // [5][TY][CX]
  static constexpr int OFF_FY = OFF_FX + 5 * TY * CX;               // [5][CY][TX]
  static constexpr int OFF_XR = OFF_FY + 5 * CY * TX;               // [4][TY][CX]
  static constexpr int OFF_YC = OFF_XR + 4 * TY * CX;               // [4][CY][TX]
  static constexpr int TOTAL = OFF_YC + 4 * CY * TX;
};

template <typename S>
inline size_t fused_smem_bytes(int TX, int TY) {
  // the window, the flux and derivative arrays; at the end the window is the
  // reduction scratch (kNumStat * (NT + 1) doubles)
  const size_t CX = TX + 4, CY = TY + 4, CELLS = CX * CY;
  const size_t win = ((kWinPlanes * 3 + kWinT + kWinR * 2) * CELLS + 9 * (size_t)TY * CX + 9 * CY * TX) * sizeof(S);
  const size_t red = (size_t)kNumStat * ((TX * TY > 256 ? 512 : 256) + 1) * sizeof(double);
  return win > red ? win : red;
}

__device__ __forceinline__ int wrapc(int c, int n) { return c < 0 ? c + n : (c >= n ? c - n : c); }

// Geometry of one CTA: tile origin, PE of the tile (z: of the chunk), PE origin.
struct FusedGeo {
  int x0, y0, pe[3], base[3];
  __device__ __forceinline__ bool beyond(const Geom& g, int d, int c) const {
    if (g.pes[d] == 1) return false;
    const int l = c - base[d];
    return l < 0 || l >= g.nl[d];
  }
  __device__ __forceinline__ int ghost_slot(const Geom& g, int d, int c) const {
    const int l = c - base[d];
    return l < 0 ? l + 2 : 2 + (l - g.nl[d]);
  }
};

// Raw values of one window plane for this thread's cells: the conserved
// variables (kind 1), the AT ghost u, v, w, T (kind 2) or nothing (kind 0:
// corner cells beyond two faces, planes beyond the z ghosts).  Fetching a
// plane into registers one iteration ahead keeps its global loads in flight
// while the current plane is computed.
template <typename S, int TX, int TY>
struct PlaneRaw {
  static constexpr int ITER = (TileShape<TX, TY>::CELLS + TileShape<TX, TY>::THREADS - 1) / TileShape<TX, TY>::THREADS;
  S v[ITER][5];
  int kind[ITER];
};

template <typename S, int TX, int TY>
__device__ __forceinline__ void fused_fetch_plane(const Geom& g, const StepArgs<S>& A, const S* __restrict__ U,
                                                  const FusedGeo& F, int zp, PlaneRaw<S, TX, TY>& P) {
  using T_ = TileShape<TX, TY>;
  const int tid = threadIdx.y * TX + threadIdx.x;
  const long long N = g.npts;
  const bool bz = F.beyond(g, 2, zp);
  const int lz = zp - F.base[2];
  const bool zfar = bz && (lz < -2 || lz >= g.nl[2] + 2);
#pragma unroll
  for (int it = 0; it < P.ITER; ++it) {
    const int c = it * T_::THREADS + tid;
    P.kind[it] = 0;
#pragma unroll
    for (int q = 0; q < 5; ++q) P.v[it][q] = S(0);
    if (c >= T_::CELLS) continue;
    const int cy = c / T_::CX, cx = c - cy * T_::CX;
    const int xg = F.x0 - 2 + cx, yg = F.y0 - 2 + cy;
    const bool bx = F.beyond(g, 0, xg), by = F.beyond(g, 1, yg);
    const S* gh = nullptr;
    long long gi = 0, qs = 0;
    if (bz) {
      if (!zfar && !bx && !by) {
        const int xw = wrapc(xg, g.n[0]), yw = wrapc(yg, g.n[1]);
        gh = A.GH[2];
        qs = 4LL * g.pes[2] * g.plane[2];
        gi = (long long)(4 * F.pe[2] + F.ghost_slot(g, 2, zp)) * g.plane[2] + (long long)yw * g.n[0] + xw;
      }
    } else if (bx) {
      if (!by) {
        const int yw = wrapc(yg, g.n[1]), zw = wrapc(zp, g.n[2]);
        gh = A.GH[0];
        qs = 4LL * g.pes[0] * g.plane[0];
        gi = (long long)(4 * F.pe[0] + F.ghost_slot(g, 0, xg)) * g.plane[0] + (long long)zw * g.n[1] + yw;
      }
    } else if (by) {
      const int xw = wrapc(xg, g.n[0]), zw = wrapc(zp, g.n[2]);
      gh = A.GH[1];
      qs = 4LL * g.pes[1] * g.plane[1];
      gi = (long long)(4 * F.pe[1] + F.ghost_slot(g, 1, yg)) * g.plane[1] + (long long)zw * g.n[0] + xw;
    } else {
      const int xw = wrapc(xg, g.n[0]), yw = wrapc(yg, g.n[1]), zw = wrapc(zp, g.n[2]);
      const long long idx = ((long long)zw * g.n[1] + yw) * g.n[0] + xw;
#pragma unroll
      for (int q = 0; q < 5; ++q) P.v[it][q] = U[q * N + idx];
      P.kind[it] = 1;
    }
    if (gh) {
#pragma unroll
      for (int q = 0; q < 4; ++q) P.v[it][q] = gh[(5 + q) * qs + gi];
      P.kind[it] = 2;
    }
  }
}

// Window plane from fetched raw values: u, v, w, T, rho and H from the
// conserved variables, or the ghost values as they are; bA, bT, bR are the
// element offsets of the plane's slots in the three window regions.
template <typename S, int TX, int TY>
__device__ __forceinline__ void fused_store_plane(const Coef<S>& K, const PlaneRaw<S, TX, TY>& P, S* win, int bA,
                                                  int bT, int bR) {
  using T_ = TileShape<TX, TY>;
  const int tid = threadIdx.y * TX + threadIdx.x;
#pragma unroll
  for (int it = 0; it < P.ITER; ++it) {
    const int c = it * T_::THREADS + tid;
    if (c >= T_::CELLS) break;
    S u = S(0), v = S(0), w = S(0), T = S(0), r = S(0), H = S(0);
    if (P.kind[it] == 1) {
      r = P.v[it][0];
      const S m0 = P.v[it][1], m1 = P.v[it][2], m2 = P.v[it][3], E = P.v[it][4];
      const S inv = rcp_rn(r);
      u = m0 * inv;
      v = m1 * inv;
      w = m2 * inv;
      const S p = pressure(K, m0, m1, m2, u, v, w, E);
      T = K.gamma * p * inv;
      H = K.eform ? E : E + p;
    } else if (P.kind[it] == 2) {
      u = P.v[it][0];
      v = P.v[it][1];
      w = P.v[it][2];
      T = P.v[it][3];
    }
    win[bA + c] = u;
    win[bA + T_::CELLS + c] = v;
    win[bA + 2 * T_::CELLS + c] = w;
    win[bT + c] = T;
    win[bR + c] = r;
    win[bR + T_::CELLS + c] = H;
  }
}

// Slots of a window plane: `q` counts planes from the chunk's first window
// plane (z_start - 4), so it is never negative (unsigned remainder); each
// region is a ring of its own depth.
template <int TX, int TY>
__device__ __forceinline__ int slot_A(int q) { return TileShape<TX, TY>::OFF_A + (int)((unsigned)q % (unsigned)kWinPlanes) * 3 * TileShape<TX, TY>::CELLS; }
template <int TX, int TY>
__device__ __forceinline__ int slot_T(int q) { return TileShape<TX, TY>::OFF_T + (int)((unsigned)q % (unsigned)kWinT) * TileShape<TX, TY>::CELLS; }
template <int TX, int TY>
__device__ __forceinline__ int slot_R(int q) { return TileShape<TX, TY>::OFF_R + (int)((unsigned)q % (unsigned)kWinR) * 2 * TileShape<TX, TY>::CELLS; }

// Fill window plane q (plane z_start - 4 + q).
template <typename S, int TX, int TY>
__device__ __forceinline__ void fused_load_plane(const Geom& g, const Coef<S>& K, const StepArgs<S>& A,
                                                 const S* __restrict__ U, const FusedGeo& F, S* win, int q,
                                                 int zp) {
  PlaneRaw<S, TX, TY> P;
  fused_fetch_plane<S, TX, TY>(g, A, U, F, zp, P);
  fused_store_plane<S, TX, TY>(K, P, win, slot_A<TX, TY>(q), slot_T<TX, TY>(q), slot_R<TX, TY>(q));
}

// The five inviscid flux components of direction d of one window cell (aA,
// aT, aR: element offsets of the cell in its plane's slots): rho u_d,
// rho u_i u_d + p delta_id, H u_d, with p = rho T / gamma.  The cell's values
// are read once for all five.
template <typename S, int TX, int TY>
__device__ __forceinline__ void cell_fluxes(const Coef<S>& K, const S* win, int aA, int aT, int aR, int d,
                                            S (&f)[5]) {
  using T_ = TileShape<TX, TY>;
  const S r = win[aR];
  const S H = win[aR + T_::CELLS];
  const S u[3] = {win[aA], win[aA + T_::CELLS], win[aA + 2 * T_::CELLS]};
  const S ud = u[d];
  const S rud = r * ud;
  f[0] = rud;
#pragma unroll
  for (int i = 0; i < 3; ++i) f[1 + i] = i == d ? fma(rud, ud, r * win[aT] * K.inv_gamma) : rud * u[i];
  f[4] = H * ud;
}

// First tap (offset from the point) of the PE-local stencil of each kind.
__device__ __forceinline__ constexpr int local_first(int kind) {
  return kind == 0 ? -2 : (kind == 1 ? 0 : (kind == 2 ? -1 : (kind == 3 ? -3 : -4)));
}

// 12 dx times the PE-local first-derivative stencil of kind KIND (Sec. 2.1),
// taps in ascending offset from local_first(KIND), applied to dv(offset).
template <int KIND, typename S, typename DV>
__device__ __forceinline__ S local_taps_c(DV dv) {
  constexpr float c[5][5] = {{1, -8, 0, 8, -1}, {-25, 48, -36, 16, -3}, {-3, -10, 18, -6, 1},
                             {-1, 6, -18, 10, 3}, {3, -16, 36, -48, 25}};
  if constexpr (KIND == 0) {
    return fma(S(8), dv(1) - dv(-1), dv(-2) - dv(2));
  } else {
    S acc = S(0);
#pragma unroll
    for (int i = 0; i < 5; ++i) acc = fma(S(c[KIND][i]), dv(local_first(KIND) + i), acc);
    return acc;
  }
}

// PE-local first-derivative stencil kind of the Sec. 2.1 mixed rule at local
// index li of a direction with nl points: 0 central, 1 first point, 2 second,
// 3 second to last, 4 last point of the PE.
__device__ __forceinline__ int local_kind(int pes, int li, int nl) {
  if (pes == 1 || (li >= 2 && li <= nl - 3)) return 0;
  if (li == 0) return 1;
  if (li == 1) return 2;
  if (li == nl - 2) return 3;
  return 4;
}

// The window seen from one point: element offsets of the point's cell in the
// u, v, w planes z-4 .. z+4, the T planes z-2 .. z+2 and the rho, H plane z,
// so that a value at (dx, dy, dz) of a field is one load at a constant offset.
template <typename S, int TX, int TY>
struct PointWin {
  using T_ = TileShape<TX, TY>;
  const S* win;                 // the shared-memory window
  int pA[kWinPlanes];           // u (v, w at + CELLS, + 2 CELLS) in planes z-4 .. z+4
  int pT[5];                    // T in planes z-2 .. z+2
  int pR;                       // rho (H at + CELLS) in plane z
  int cell;                     // the point's cell within a plane
  __device__ __forceinline__ S at(int f, int dx, int dy, int dz) const {
    const int o = dy * T_::CX + dx;
    if (f <= WF_W) return win[pA[4 + dz] + f * T_::CELLS + o];
    if (f == WF_T) return win[pT[2 + dz] + o];
    return win[pR + (f - WF_R) * T_::CELLS + o];
  }
  // value shifted by m along direction d
  __device__ __forceinline__ S sh(int f, int d, int m, int dx = 0, int dy = 0, int dz = 0) const {
    return at(f, dx + (d == 0 ? m : 0), dy + (d == 1 ? m : 0), dz + (d == 2 ? m : 0));
  }
  // 12 dz times the PE-local derivative along z (stencil `kind`, uniform over
  // the CTA) of the AT derivative of u, v or w along `in` (x or y); each kind
  // is its own code path, so every tap reads a window plane at a constant slot.
  __device__ __forceinline__ S zlocal_of_d1(const Coef<S>& K, int f, int in, int kind) const {
    const int sk = in == 0 ? 1 : T_::CX;
    auto dv = [&](int o) {   // inner derivative at plane z + o
      const S* q = win + pA[4 + o] + f * T_::CELLS;
      return fma(K.c1[in], q[sk] - q[-sk], K.c2[in] * (q[2 * sk] - q[-2 * sk]));
    };
    switch (kind) {
      case 0: return local_taps_c<0, S>(dv);
      case 1: return local_taps_c<1, S>(dv);
      case 2: return local_taps_c<2, S>(dv);
      case 3: return local_taps_c<3, S>(dv);
      default: return local_taps_c<4, S>(dv);
    }
  }
};

// Five-tap PE-local stencil with the thread's own coefficients (kind fixed
// for the thread's column; registers, or a row of the shared table), taps
// STEP elements apart from q.
template <int STEP, typename S, typename C>
__device__ __forceinline__ S local_taps(const C& c, const S* q) {
  S acc = S(0);
#pragma unroll
  for (int i = 0; i < 5; ++i) acc = fma(c[i], q[i * STEP], acc);
  return acc;
}

// Per-thread statistics accumulators over the thread's column of one z chunk
// (at most 64 points).  FP64 form: plain FP64 sums.  FP32 forms: compensated
// (Kahan) FP32 sums, whose error does not grow with the number of points;
// the block reduction carries each as a double-float pair and the block's
// partial is FP64.
template <typename S>
struct StatAcc {
  S s[kNumStat];
  S c[sizeof(S) == 4 ? kNumStat : 1];   // Kahan compensations (FP32 forms)
  __device__ void init() {
#pragma unroll
    for (int i = 0; i < kNumStat; ++i) s[i] = S(0);
#pragma unroll
    for (int i = 0; i < (sizeof(S) == 4 ? kNumStat : 1); ++i) c[i] = S(0);
  }
  __device__ void add(int i, S v) {
    if constexpr (sizeof(S) == 4) {
      const S y = __fsub_rn(v, c[i]);
      const S t = __fadd_rn(s[i], y);
      c[i] = __fsub_rn(__fsub_rn(t, s[i]), y);
      s[i] = t;
    } else {
      s[i] += v;
    }
  }
};

template <typename S, int TX, int TY>
__global__ void __launch_bounds__(TX * TY, (sizeof(S) == 4 && TX * TY <= 256) ? 2 : 1)
    k_fused(Geom g, Coef<S> K, StepArgs<S> A0, int ZC) {
  const StepArgs<S>& A = A0;
  const StepDyn<S> D = resolve_step(A0);
  using T_ = TileShape<TX, TY>;
  extern __shared__ __align__(16) unsigned char fused_smem[];
  S* win = reinterpret_cast<S*>(fused_smem);
  FusedGeo F;
  F.x0 = blockIdx.x * TX;
  F.y0 = blockIdx.y * TY;
  const int zs = blockIdx.z * ZC;
  F.pe[0] = F.x0 / g.nl[0];
  F.pe[1] = F.y0 / g.nl[1];
  F.pe[2] = zs / g.nl[2];
  for (int d = 0; d < 3; ++d) F.base[d] = F.pe[d] * g.nl[d];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int x = F.x0 + tx, y = F.y0 + ty;
  const int cell = (ty + 2) * T_::CX + (tx + 2);
  const long long N = g.npts;

  // PE-local stencil coefficients (x 12) by kind, taps in ascending offset:
  // central, first point, second point, second to last, last (Sec. 2.1)
  __shared__ S coef[5][5];
  {
    const int t0 = threadIdx.y * TX + threadIdx.x;   // tiles hold at least 64 threads
    if (t0 < 25) {
      const float t[5][5] = {{1, -8, 0, 8, -1}, {-25, 48, -36, 16, -3}, {-3, -10, 18, -6, 1},
                             {-1, 6, -18, 10, 3}, {3, -16, 36, -48, 25}};
      coef[t0 / 5][t0 % 5] = S(t[t0 / 5][t0 % 5]);
    }
  }

  StatAcc<S> st;
  st.init();
  long long kwave = LLONG_MIN, krho = LLONG_MAX, kp = LLONG_MAX;
  // FP32 form: running max / min in FP32 (keys formed once at the end)
  S wmax = S(0), rmin = S(3.0e38), pmin = S(3.0e38);
  unsigned health = 0;

  const int li_x = x - F.base[0], li_y = y - F.base[1];
  const int kind_x = local_kind(g.pes[0], li_x, g.nl[0]), kind_y = local_kind(g.pes[1], li_y, g.nl[1]);
  const S a0sum = K.a0[0] + K.a0[1] + K.a0[2];
  const int tid = ty * TX + tx;
  S* FX = win + T_::OFF_FX;                    // [5][TY][CX]
  S* FY = win + T_::OFF_FY;                    // [5][CY][TX]
  S* XR = win + T_::OFF_XR;                    // [4][TY][CX]
  S* YC = win + T_::OFF_YC;                    // [4][CY][TX]
  const long long qsx = 4LL * g.pes[0] * g.plane[0], qsy = 4LL * g.pes[1] * g.plane[1];
  const long long qsz = 4LL * g.pes[2] * g.plane[2];

  // z fluxes of this column at window plane q = zp - zs + 4 (z ghosts beyond
  // a PE z-face), formed afresh each plane for z-2 .. z+2
  auto zflux = [&](int zp, int q, S (&out)[5]) {
    if (F.beyond(g, 2, zp)) {
      const long long gi = (long long)(4 * F.pe[2] + F.ghost_slot(g, 2, zp)) * g.plane[2] + (long long)y * g.n[0] + x;
#pragma unroll
      for (int e = 0; e < 5; ++e) out[e] = A.GH[2][e * qsz + gi];
    } else {
      const int aA = slot_A<TX, TY>(q) + cell, aT = slot_T<TX, TY>(q) + cell, aR = slot_R<TX, TY>(q) + cell;
      cell_fluxes<S, TX, TY>(K, win, aA, aT, aR, 2, out);
    }
  };

  // window planes q = 0 .. 7 (z = zs-4 .. zs+3)
  for (int q = 0; q < 8; ++q) fused_load_plane<S, TX, TY>(g, K, A, D.U, F, win, q, zs - 4 + q);
  __syncthreads();
  // the PE-local x- and y-stencils of this thread's column, and their first
  // taps in the x-row and y-column arrays; the x coefficients vary across a
  // warp and are kept in registers, the y ones are read from the table (one
  // row per warp where a warp spans one tile row)
  S lcx[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) lcx[i] = coef[kind_x][i];
  const S* lcy = coef[kind_y];
  const int ax0 = ty * T_::CX + tx + 2 + local_first(kind_x);
  const int ay0 = (ty + 2 + local_first(kind_y)) * TX + tx;
  PlaneRaw<S, TX, TY> pf;                       // plane z + 4, fetched one iteration ahead
  fused_fetch_plane<S, TX, TY>(g, A, D.U, F, zs + 4, pf);

  for (int z = zs; z < zs + ZC; ++z) {
    const int q = z - zs + 4;                  // window-plane count of plane z
    fused_store_plane<S, TX, TY>(K, pf, win, slot_A<TX, TY>(q + 4), slot_T<TX, TY>(q + 4), slot_R<TX, TY>(q + 4));
    __syncthreads();
    if (z + 1 < zs + ZC) fused_fetch_plane<S, TX, TY>(g, A, D.U, F, z + 5, pf);
    // the point's conserved variables and R^{n-1}: loaded here so that the
    // loads are in flight during the flux phase
    const long long idx = ((long long)z * g.n[1] + y) * g.n[0] + x;
    const S m[3] = {D.U[N + idx], D.U[2 * N + idx], D.U[3 * N + idx]};
    const S Ecur = D.U[4 * N + idx];
    S Rp[5], Lp[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) Rp[v] = needs_rprev(A, D) ? A.Rprev[v * N + idx] : S(0);
    // the compensated form's low words of U^n, loaded with R^{n-1}
#pragma unroll
    for (int v = 0; v < 5; ++v) Lp[v] = (A.do_update && D.Ulo) ? D.Ulo[v * N + idx] : S(0);
    // fluxes of the current plane (x on x-extended rows, y on y-extended
    // columns), and on the same cells the AT derivatives the mixed rule's x-
    // and y-stencils take
    {
      const int bA = slot_A<TX, TY>(q), bT = slot_T<TX, TY>(q), bR = slot_R<TX, TY>(q);
      const int bAm1 = slot_A<TX, TY>(q - 1), bAp1 = slot_A<TX, TY>(q + 1);
      const int bAm2 = slot_A<TX, TY>(q - 2), bAp2 = slot_A<TX, TY>(q + 2);
      // d/dz of field f (0 u, 2 w) at window cell cw of plane z
      auto ddz = [&](int f, int cw) {
        const int o = f * T_::CELLS + cw;
        return fma(K.c1[2], win[bAp1 + o] - win[bAm1 + o], K.c2[2] * (win[bAp2 + o] - win[bAm2 + o]));
      };
      // The cells of the last, partial pass of each loop go to warps that the
      // other loop's partial pass leaves idle (y: the top warps, x: the warps
      // just below them), so the warps reach the next barrier together; the
      // rotation is by whole warps, which keeps each warp on consecutive cells.
      constexpr int kNT = T_::THREADS;
      constexpr int kRemY = ((TY + 4) * TX % kNT + 31) / 32 * 32;
      constexpr int kRemX = (TY * T_::CX % kNT + 31) / 32 * 32;
      const int tid_x = (tid + kRemY + kRemX) % kNT, tid_y = (tid + kRemY) % kNT;
#pragma unroll
      for (int c0 = 0; c0 < TY * T_::CX; c0 += T_::THREADS) {
        const int c = c0 + tid_x;
        if (c < TY * T_::CX) {
          const int r = c / T_::CX, cxw = c - r * T_::CX;
          const int xg = F.x0 - 2 + cxw, yg = F.y0 + r;
          const int cw = (r + 2) * T_::CX + cxw;
          if (F.beyond(g, 0, xg)) {
            const long long gi = (long long)(4 * F.pe[0] + F.ghost_slot(g, 0, xg)) * g.plane[0] +
                                 (long long)z * g.n[1] + yg;
#pragma unroll
            for (int e = 0; e < 5; ++e) FX[e * TY * T_::CX + c] = A.GH[0][e * qsx + gi];
          } else {
            S f[5];
            cell_fluxes<S, TX, TY>(K, win, bA + cw, bT + cw, bR + cw, 0, f);
#pragma unroll
            for (int e = 0; e < 5; ++e) FX[e * TY * T_::CX + c] = f[e];
          }
          // (cells beyond the x-face are never read by the PE-local x-stencils)
          const S* vq = win + bA + T_::CELLS + cw;
          const S* uq = win + bA + cw;
          XR[XR_VY * TY * T_::CX + c] = fma(K.c1[1], vq[T_::CX] - vq[-T_::CX], K.c2[1] * (vq[2 * T_::CX] - vq[-2 * T_::CX]));
          XR[XR_UY * TY * T_::CX + c] = fma(K.c1[1], uq[T_::CX] - uq[-T_::CX], K.c2[1] * (uq[2 * T_::CX] - uq[-2 * T_::CX]));
          XR[XR_WZ * TY * T_::CX + c] = ddz(2, cw);
          XR[XR_UZ * TY * T_::CX + c] = ddz(0, cw);
        }
      }
#pragma unroll
      for (int c0 = 0; c0 < (TY + 4) * TX; c0 += T_::THREADS) {
        const int c = c0 + tid_y;
        if (c < (TY + 4) * TX) {
          const int r = c / TX, cxl = c - r * TX;
          const int xg = F.x0 + cxl, yg = F.y0 - 2 + r;
          const int cw = r * T_::CX + cxl + 2;
          if (F.beyond(g, 1, yg)) {
            const long long gi = (long long)(4 * F.pe[1] + F.ghost_slot(g, 1, yg)) * g.plane[1] +
                                 (long long)z * g.n[0] + xg;
#pragma unroll
            for (int e = 0; e < 5; ++e) FY[e * (TY + 4) * TX + c] = A.GH[1][e * qsy + gi];
          } else {
            S f[5];
            cell_fluxes<S, TX, TY>(K, win, bA + cw, bT + cw, bR + cw, 1, f);
#pragma unroll
            for (int e = 0; e < 5; ++e) FY[e * (TY + 4) * TX + c] = f[e];
          }
          const S* vq = win + bA + T_::CELLS + cw;
          const S* uq = win + bA + cw;
          YC[YC_VX * (TY + 4) * TX + c] = fma(K.c1[0], vq[1] - vq[-1], K.c2[0] * (vq[2] - vq[-2]));
          YC[YC_UX * (TY + 4) * TX + c] = fma(K.c1[0], uq[1] - uq[-1], K.c2[0] * (uq[2] - uq[-2]));
          YC[YC_WZ * (TY + 4) * TX + c] = ddz(2, cw);
          YC[YC_VZ * (TY + 4) * TX + c] = ddz(1, cw);
        }
      }
    }
    __syncthreads();
    PointWin<S, TX, TY> W;
    W.win = win;
    W.cell = cell;
#pragma unroll
    for (int k = 0; k < kWinPlanes; ++k) W.pA[k] = slot_A<TX, TY>(q - 4 + k) + cell;
#pragma unroll
    for (int k = 0; k < 5; ++k) W.pT[k] = slot_T<TX, TY>(q - 2 + k) + cell;
    W.pR = slot_R<TX, TY>(q) + cell;
    const int li_z = z - F.base[2];
    const int kind_z = local_kind(g.pes[2], li_z, g.nl[2]);

    // ---- inviscid flux divergence: -sum_d D_d F_d (ghost fluxes already in
    // the flux arrays / queue across PE faces)
    S dz1[5], dz2[5];   // F_z(z+1) - F_z(z-1), F_z(z+2) - F_z(z-2) of this column
    {
      S fa[5], fb[5];
      zflux(z + 1, q + 1, fa);
      zflux(z - 1, q - 1, fb);
#pragma unroll
      for (int e = 0; e < 5; ++e) dz1[e] = fa[e] - fb[e];
      zflux(z + 2, q + 2, fa);
      zflux(z - 2, q - 2, fb);
#pragma unroll
      for (int e = 0; e < 5; ++e) dz2[e] = fa[e] - fb[e];
    }
    S R[5];
#pragma unroll
    for (int e = 0; e < 5; ++e) {
      const S* fx = FX + e * TY * T_::CX + ty * T_::CX + tx + 2;
      const S* fy = FY + e * (TY + 4) * TX + (ty + 2) * TX + tx;
      S acc = S(0);
      acc = fma(-K.c1[0], fx[1] - fx[-1], acc);
      acc = fma(-K.c2[0], fx[2] - fx[-2], acc);
      acc = fma(-K.c1[1], fy[TX] - fy[-TX], acc);
      acc = fma(-K.c2[1], fy[2 * TX] - fy[-2 * TX], acc);
      acc = fma(-K.c1[2], dz1[e], acc);
      acc = fma(-K.c2[2], dz2[e], acc);
      R[e] = acc;
    }

    // ---- second derivatives of u, v, w, T; first derivatives at the point
    S lap[4], d2diag[3], Ag[3][3], dT[3];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const S f0 = W.at(WF_U + q, 0, 0, 0);
      S accq = a0sum * f0;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const S fm2 = W.sh(WF_U + q, d, -2), fm1 = W.sh(WF_U + q, d, -1);
        const S fp1 = W.sh(WF_U + q, d, 1), fp2 = W.sh(WF_U + q, d, 2);
        const S off = fma(K.a1[d], fp1 + fm1, K.a2[d] * (fp2 + fm2));
        accq += off;
        if (q == d) d2diag[d] = fma(K.a0[d], f0, off);
        const S d1 = fma(K.c1[d], fp1 - fm1, K.c2[d] * (fp2 - fm2));
        if (q < 3) Ag[q][d] = d1; else dT[d] = d1;
      }
      lap[q] = accq;
    }

    // ---- d theta/dx_i = d2 u_i/dx_i^2 + sum_{k != i} d/dx_i (d u_k/dx_k), the
    // mixed terms by the three-step rule (Sec. 2.1): part a is the PE-local
    // derivative along a of the AT derivative along b, part b the one along b
    // of the derivative along a; inside both stencils' reach the term is the
    // central part a, elsewhere the average of the two parts
    S gth[3];
    {
      const int sxr = TY * T_::CX, syc = (TY + 4) * TX;
      auto mix = [&](S pa, S pb, bool bnd) { return bnd ? S(0.5) * (pa + pb) : pa; };
      const bool bxy = kind_x != 0 || kind_y != 0, bxz = kind_x != 0 || kind_z != 0, byz = kind_y != 0 || kind_z != 0;
      auto tx_ = [&](int fld) { return local_taps<1>(lcx, XR + fld * sxr + ax0); };
      auto ty_ = [&](int fld) { return local_taps<TX>(lcy, YC + fld * syc + ay0); };
      // d/dx (dv/dy)
      const S m_xy = mix(K.hloc[0] * tx_(XR_VY), K.hloc[1] * ty_(YC_VX), bxy);
      // d/dy (du/dx)
      const S m_yx = mix(K.hloc[1] * ty_(YC_UX), K.hloc[0] * tx_(XR_UY), bxy);
      // d/dx (dw/dz): part b along z needs the window (planes z-4 .. z+4)
      const S pa_xz = K.hloc[0] * tx_(XR_WZ);
      const S pb_xz = __any_sync(__activemask(), bxz) ? K.hloc[2] * W.zlocal_of_d1(K, WF_W, 0, kind_z) : S(0);
      // d/dz (du/dx)
      const S pa_zx = K.hloc[2] * W.zlocal_of_d1(K, WF_U, 0, kind_z);
      const S pb_zx = K.hloc[0] * tx_(XR_UZ);
      // d/dy (dw/dz)
      const S pa_yz = K.hloc[1] * ty_(YC_WZ);
      const S pb_yz = __any_sync(__activemask(), byz) ? K.hloc[2] * W.zlocal_of_d1(K, WF_W, 1, kind_z) : S(0);
      // d/dz (dv/dy)
      const S pa_zy = K.hloc[2] * W.zlocal_of_d1(K, WF_V, 1, kind_z);
      const S pb_zy = K.hloc[1] * ty_(YC_VZ);
      gth[0] = d2diag[0] + m_xy + mix(pa_xz, pb_xz, bxz);
      gth[1] = d2diag[1] + m_yx + mix(pa_yz, pb_yz, byz);
      gth[2] = d2diag[2] + mix(pa_zx, pb_zx, bxz) + mix(pa_zy, pb_zy, byz);
    }

    // ---- point values
    const S r = W.at(WF_R, 0, 0, 0);
    const S vel[3] = {W.at(WF_U, 0, 0, 0), W.at(WF_V, 0, 0, 0), W.at(WF_W, 0, 0, 0)};
    const S T = W.at(WF_T, 0, 0, 0);
    const S p = pressure(K, m[0], m[1], m[2], vel[0], vel[1], vel[2], Ecur);
    const S theta = Ag[0][0] + Ag[1][1] + Ag[2][2];
    S mu, dmudT;
    viscosity(K, T, mu, dmudT);
    const S kappa = mu * K.cp_over_pr;
    S dmu[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) dmu[j] = dmudT * dT[j];
    S sm[3][3];
    const S th23 = S(2.0 / 3.0) * theta;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) sm[i][j] = i == j ? S(2) * Ag[i][i] - th23 : Ag[i][j] + Ag[j][i];

    S fo[3] = {S(0), S(0), S(0)};
    if (A.fB) {
      const long long lines = (long long)g.n[2] * g.n[1];
      const long long ln = (long long)z * g.n[1] + y;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        S acc = S(0);
        for (int kx = 0; kx <= A.fK; ++kx) {
          const vec2_t<S> b = A.fB[((long long)kx * 3 + c) * lines + ln];
          const vec2_t<S> e = A.fX[(long long)kx * g.n[0] + x];
          acc = fma(b.x, e.x, fma(-b.y, e.y, acc));
        }
        fo[c] = acc;
      }
    }

    S sS = sm[0][0] * Ag[0][0] + sm[1][1] * Ag[1][1] + sm[2][2] * Ag[2][2];
    sS = fma(sm[0][1], sm[0][1], sS);
    sS = fma(sm[0][2], sm[0][2], sS);
    sS = fma(sm[1][2], sm[1][2], sS);
    const S sigS = mu * sS;
    S work = S(0);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      S V = mu * fma(gth[i], S(1.0 / 3.0), lap[i]);
#pragma unroll
      for (int j = 0; j < 3; ++j) V = fma(dmu[j], sm[i][j], V);
      R[1 + i] += fma(r, fo[i], V);
      work = fma(vel[i], V, work);
    }
    const S heat = fma(K.cp_over_pr, fma(dmu[0], dT[0], fma(dmu[1], dT[1], dmu[2] * dT[2])), kappa * lap[3]);
    if (K.eform) R[4] += fma(-p, theta, sigS + heat);
    else R[4] += fma(r, fma(fo[0], vel[0], fma(fo[1], vel[1], fo[2] * vel[2])), sigS + work + heat);

    if (nonpositive(r)) health |= H_RHO;
    if (nonpositive(p)) health |= H_P;
#pragma unroll
    for (int v = 0; v < 5; ++v)
      if (nonfinite(R[v])) health |= H_NONFINITE;

    if (A.do_update) {
      const S Uo[5] = {r, m[0], m[1], m[2], Ecur};
      S un[5], unlo[5];
      ab2_update(K, A, D, idx, N, Uo, R, un, unlo, health, Rp, D.Ulo ? Lp : nullptr);
      // (the ring slabs of level n+1 are written by the next step's ghost kernel)
      stage_xface(g, A, li_x, F.pe[0], (long long)z * g.n[1] + y, un, unlo);
    } else if (A.Rout) {
#pragma unroll
      for (int v = 0; v < 5; ++v) A.Rout[v * N + idx] = (double)R[v];
    }

    if (A.do_stats) {
      const S uu = fma(vel[0], vel[0], fma(vel[1], vel[1], vel[2] * vel[2]));
      const S c = sqrt(T);
      st.add(ST_RHO, r);
      st.add(ST_M0, m[0]);
      st.add(ST_M1, m[1]);
      st.add(ST_M2, m[2]);
      st.add(ST_E, Ecur);
      st.add(ST_KE, S(0.5) * r * uu);
      st.add(ST_SIGS, sigS);
      const S a0 = Ag[0][0], a1 = Ag[1][1], a2 = Ag[2][2];
      const S q0 = a0 * a0, q1 = a1 * a1, q2 = a2 * a2;
      st.add(ST_G2, q0 + q1 + q2);
      st.add(ST_G3, fma(q0, a0, fma(q1, a1, q2 * a2)));
      st.add(ST_G4, fma(q0, q0, fma(q1, q1, q2 * q2)));
      const S o0 = Ag[2][1] - Ag[1][2], o1 = Ag[0][2] - Ag[2][0], o2 = Ag[1][0] - Ag[0][1];
      st.add(ST_ENST, fma(o0, o0, fma(o1, o1, o2 * o2)));
      st.add(ST_PTHETA, p * theta);
      st.add(ST_FPOW, r * fma(fo[0], vel[0], fma(fo[1], vel[1], fo[2] * vel[2])));
      st.add(ST_U2, uu);
      st.add(ST_C, c);
      const S au[3] = {fabs(vel[0]), fabs(vel[1]), fabs(vel[2])};
      if constexpr (sizeof(S) == 4) {
        wmax = fmaxf(wmax, fmaxf(fmaxf(au[0], au[1]), au[2]) + c);
        rmin = fminf(rmin, r);
        pmin = fminf(pmin, p);
      } else {
        const long long k0 = okey(au[0]), k1 = okey(au[1]), k2 = okey(au[2]);
        const S umax = (k0 >= k1 && k0 >= k2) ? au[0] : (k1 >= k2 ? au[1] : au[2]);
        kwave = max(kwave, okey(umax + c));
        krho = min(krho, okey(r));
        kp = min(kp, okey(p));
      }
    }
    __syncthreads();
  }
  // the window is dead after the last barrier: reuse it as reduction scratch
  if constexpr (sizeof(S) == 4) {
    if (A.do_stats) {
      kwave = okey(wmax);
      krho = okey(rmin);
      kp = okey(pmin);
    }
    block_reduce<S, (TX * TY > 256 ? 512 : 256)>(st.s, kwave, krho, kp, health, A.do_stats != 0, A.partial, A.words,
                                                 reinterpret_cast<double*>(fused_smem), st.c);
  } else {
    block_reduce<S, (TX * TY > 256 ? 512 : 256)>(st.s, kwave, krho, kp, health, A.do_stats != 0, A.partial, A.words,
                                                 reinterpret_cast<double*>(fused_smem));
  }
}

}  // namespace atdns
