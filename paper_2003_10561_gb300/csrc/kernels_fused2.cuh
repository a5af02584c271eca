// Fused AT-DNS step kernel, paired form (FP32-bulk forms only).
//
// The same single pass over U as k_fused (kernels_fused.cuh): a CTA owns a
// TX x TY tile of one PE and marches z through a chunk of ZC planes with the
// same shared-memory window (u, v, w for nine planes, T, rho, H for seven,
// AT ghost values beyond PE faces), per-plane x / y flux arrays and per-plane
// arrays of the AT derivatives the mixed rule's x- and y-stencils take, and
// the same arithmetic per point (Sec. 2, Sec. 2.1, Eq. (time_ab)).
//
// What differs: each thread owns two x-adjacent points (TX/2 threads per tile
// row) and carries them as float2 pairs through the packed FP32 instructions
// of sm_100+ (one instruction computes both lanes of a pair), so the
// instruction count per point -- the bound of this kernel -- roughly halves:
//   * every window, flux and derivative-array access of a pair is one 64-bit
//     shared-memory load (cells of a pair are adjacent and 8-byte aligned:
//     tiles start at even x and every row holds an even number of cells);
//   * y- and z-stencils are packed arithmetic on those pairs;
//   * x-stencils of a pair take the six cells x-2 .. x+3 from three aligned
//     64-bit loads; the odd-offset differences are two scalar operations;
//   * the window fill, the flux phase and the per-plane derivative arrays
//     work on cell pairs too (a PE face never splits a pair: PE extents are
//     multiples of 8).
// The mixed rule's PE-local x-stencils of a pair run over a six-cell window
// starting at an even cell with per-point coefficients padded with zeros
// (central pairs, the first two points and the last two points of a PE row
// each fit one such window).
#pragma once
#include <type_traits>

#include "kernels_fused.cuh"

namespace atdns {

using f2 = float2;

__device__ __forceinline__ f2 pk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ f2 bc(float a) { return make_float2(a, a); }
__device__ __forceinline__ f2 operator+(f2 a, f2 b) { return __fadd2_rn(a, b); }
// a - b = fma(b, -1, a): one packed instruction, rounded once like a subtraction
__device__ __forceinline__ f2 operator-(f2 a, f2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ f2 operator*(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ f2 ld2(const float* p) { return *reinterpret_cast<const f2*>(p); }
__device__ __forceinline__ void st2(float* p, f2 v) { *reinterpret_cast<f2*>(p) = v; }
__device__ __forceinline__ f2 rcp2(f2 a) { return pk(rcp_rn(a.x), rcp_rn(a.y)); }

template <int TX, int TY>
struct PairShape {
  static constexpr int TXH = TX / 2;                  // threads per tile row
  static constexpr int NT = TXH * TY;                 // threads of a CTA
  static constexpr int CX = TX + 4, CY = TY + 4, CELLS = CX * CY;
  // window fill items of one plane: the tile's own columns of every window
  // row as aligned quads of 4 cells (x0 + 4j: one 128-bit load per variable),
  // then the two x-halo cell pairs of every row (x0 - 2 and x0 + TX)
  static constexpr int QROW = TX / 4, NQ = QROW * CY, NH = 2 * CY;
  static constexpr int ITEMS = NQ + NH;
  static constexpr int ITER = (ITEMS + NT - 1) / NT;
  static_assert(TX % 16 == 0 && TY % 8 == 0, "paired tiles are 16 or 32 wide and a multiple of 8 high");
};

// Raw values of one window plane for this thread's fill items (a quad in
// x, y, z, w of each variable, or a pair in x, y; kind 1: the conserved
// variables, 2: AT ghost u, v, w, T, 0: nothing).
template <int TX, int TY>
struct PlaneRaw2 {
  float4 v[PairShape<TX, TY>::ITER][5];
  int kind[PairShape<TX, TY>::ITER];
};

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }

template <int TX, int TY>
__device__ __forceinline__ void fetch_plane2(const Geom& g, const StepArgs<float>& A, const float* __restrict__ U,
                                             const FusedGeo& F, int zp, PlaneRaw2<TX, TY>& P) {
  using PS = PairShape<TX, TY>;
  const int tid = threadIdx.x;
  const long long N = g.npts;
  const bool bz = F.beyond(g, 2, zp);
  const int lz = zp - F.base[2];
  const bool zfar = bz && (lz < -2 || lz >= g.nl[2] + 2);
  const int zw = wrapc(zp, g.n[2]);
#pragma unroll
  for (int it = 0; it < PS::ITER; ++it) {
    const int i = it * PS::NT + tid;
    P.kind[it] = 0;
#pragma unroll
    for (int q = 0; q < 5; ++q) P.v[it][q] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i >= PS::ITEMS) continue;
    if (i < PS::NQ) {
      // a quad of the tile's own columns: never beyond an x-face (tiles lie in one PE)
      const int cy = i / PS::QROW, j = i - cy * PS::QROW;
      const int xg = F.x0 + 4 * j, yg = F.y0 - 2 + cy;
      const bool by = F.beyond(g, 1, yg);
      if (bz) {
        if (!zfar && !by) {
          const int yw = wrapc(yg, g.n[1]);
          const long long qs = 4LL * g.pes[2] * g.plane[2];
          const long long gi = checked((long long)(4 * F.pe[2] + F.ghost_slot(g, 2, zp)) * g.plane[2] +
                                           (long long)yw * g.n[0] + xg, qs - 3, A.ds, CHK_GHOST);
#pragma unroll
          for (int q = 0; q < 4; ++q) P.v[it][q] = ld4(A.GH[2] + (5 + q) * qs + gi);
          P.kind[it] = 2;
        }
      } else if (by) {
        const long long qs = 4LL * g.pes[1] * g.plane[1];
        const long long gi = checked((long long)(4 * F.pe[1] + F.ghost_slot(g, 1, yg)) * g.plane[1] +
                                         (long long)zw * g.n[0] + xg, qs - 3, A.ds, CHK_GHOST);
#pragma unroll
        for (int q = 0; q < 4; ++q) P.v[it][q] = ld4(A.GH[1] + (5 + q) * qs + gi);
        P.kind[it] = 2;
      } else {
        const int yw = wrapc(yg, g.n[1]);
        const long long idx = checked(((long long)zw * g.n[1] + yw) * g.n[0] + xg, N - 3, A.ds, CHK_STATE);
#pragma unroll
        for (int q = 0; q < 5; ++q) P.v[it][q] = ld4(U + q * N + idx);
        P.kind[it] = 1;
      }
      continue;
    }
    // an x-halo pair of a window row
    const int h = i - PS::NQ, cy = h >> 1;
    const int xg = (h & 1) ? F.x0 + TX : F.x0 - 2, yg = F.y0 - 2 + cy;   // xg is even: the pair is xg, xg + 1
    const bool bx = F.beyond(g, 0, xg), by = F.beyond(g, 1, yg);
    auto put = [&](int q, f2 w) { P.v[it][q].x = w.x; P.v[it][q].y = w.y; };
    if (bz) {
      if (!zfar && !bx && !by) {
        const int xw = wrapc(xg, g.n[0]), yw = wrapc(yg, g.n[1]);
        const long long qs = 4LL * g.pes[2] * g.plane[2];
        const long long gi = checked((long long)(4 * F.pe[2] + F.ghost_slot(g, 2, zp)) * g.plane[2] +
                                         (long long)yw * g.n[0] + xw, qs - 1, A.ds, CHK_GHOST);
#pragma unroll
        for (int q = 0; q < 4; ++q) put(q, ld2(A.GH[2] + (5 + q) * qs + gi));
        P.kind[it] = 2;
      }
    } else if (bx) {
      if (!by) {
        // the two cells are consecutive ghost slots of the x-face
        const int yw = wrapc(yg, g.n[1]);
        const long long qs = 4LL * g.pes[0] * g.plane[0];
        const long long g0 = checked((long long)(4 * F.pe[0] + F.ghost_slot(g, 0, xg)) * g.plane[0] +
                                         (long long)zw * g.n[1] + yw, qs - g.plane[0], A.ds, CHK_GHOST);
        const long long g1 = g0 + g.plane[0];
#pragma unroll
        for (int q = 0; q < 4; ++q) put(q, pk(A.GH[0][(5 + q) * qs + g0], A.GH[0][(5 + q) * qs + g1]));
        P.kind[it] = 2;
      }
    } else if (by) {
      const int xw = wrapc(xg, g.n[0]);
      const long long qs = 4LL * g.pes[1] * g.plane[1];
      const long long gi = checked((long long)(4 * F.pe[1] + F.ghost_slot(g, 1, yg)) * g.plane[1] +
                                       (long long)zw * g.n[0] + xw, qs - 1, A.ds, CHK_GHOST);
#pragma unroll
      for (int q = 0; q < 4; ++q) put(q, ld2(A.GH[1] + (5 + q) * qs + gi));
      P.kind[it] = 2;
    } else {
      const int xw = wrapc(xg, g.n[0]), yw = wrapc(yg, g.n[1]);
      const long long idx = checked(((long long)zw * g.n[1] + yw) * g.n[0] + xw, N - 1, A.ds, CHK_STATE);
#pragma unroll
      for (int q = 0; q < 5; ++q) put(q, ld2(U + q * N + idx));
      P.kind[it] = 1;
    }
  }
}

// Window quantities of one cell pair from its raw values: u, v, w, T, rho, H
// (zeros for kind 0; rho = H = 0 at ghost cells, whose fluxes come from the
// ghost arrays).
template <bool PLAIN>
__device__ __forceinline__ void store_cells2(const Coef<float>& K, const CoefPair& KP, int kind, f2 r0, f2 m0, f2 m1,
                                             f2 m2, f2 E, float* win, int bA, int bT, int bR, int c, int CELLS) {
  const bool eform = !PLAIN && K.eform;
  f2 u = bc(0.f), v = bc(0.f), w = bc(0.f), T = bc(0.f), r = bc(0.f), H = bc(0.f);
  if (kind == 1) {
    r = r0;
    const f2 inv = rcp2(r);
    u = m0 * inv;
    v = m1 * inv;
    w = m2 * inv;
    // (gamma-1)(E - (m.u)/2), or (gamma-1) rho e
    const f2 p_ = eform ? KP.gm1 * E : KP.gm1 * fma2(bc(-0.5f), fma2(m0, u, fma2(m1, v, m2 * w)), E);
    T = KP.gamma * p_ * inv;
    H = eform ? E : E + p_;
  } else if (kind == 2) {
    u = r0;
    v = m0;
    w = m1;
    T = m2;
  }
  st2(win + bA + c, u);
  st2(win + bA + CELLS + c, v);
  st2(win + bA + 2 * CELLS + c, w);
  st2(win + bT + c, T);
  st2(win + bR + c, r);
  st2(win + bR + CELLS + c, H);
}

template <int TX, int TY, bool PLAIN>
__device__ __forceinline__ void store_plane2(const Coef<float>& K, const CoefPair& KP, const PlaneRaw2<TX, TY>& P,
                                             float* win, int bA, int bT, int bR) {
  using PS = PairShape<TX, TY>;
  const int tid = threadIdx.x;
#pragma unroll
  for (int it = 0; it < PS::ITER; ++it) {
    const int i = it * PS::NT + tid;
    if (i >= PS::ITEMS) break;
    const float4* x = P.v[it];
    if (i < PS::NQ) {
      const int cy = i / PS::QROW, j = i - cy * PS::QROW;
      const int c = cy * PS::CX + 2 + 4 * j;
      store_cells2<PLAIN>(K, KP, P.kind[it], pk(x[0].x, x[0].y), pk(x[1].x, x[1].y), pk(x[2].x, x[2].y),
                          pk(x[3].x, x[3].y), pk(x[4].x, x[4].y), win, bA, bT, bR, c, PS::CELLS);
      store_cells2<PLAIN>(K, KP, P.kind[it], pk(x[0].z, x[0].w), pk(x[1].z, x[1].w), pk(x[2].z, x[2].w),
                          pk(x[3].z, x[3].w), pk(x[4].z, x[4].w), win, bA, bT, bR, c + 2, PS::CELLS);
    } else {
      const int h = i - PS::NQ, cy = h >> 1;
      const int c = cy * PS::CX + ((h & 1) ? TX + 2 : 0);
      store_cells2<PLAIN>(K, KP, P.kind[it], pk(x[0].x, x[0].y), pk(x[1].x, x[1].y), pk(x[2].x, x[2].y),
                          pk(x[3].x, x[3].y), pk(x[4].x, x[4].y), win, bA, bT, bR, c, PS::CELLS);
    }
  }
}

// The five inviscid flux components of direction d of a cell pair (element
// offsets of the pair's first cell in its plane's slots).
template <int TX, int TY>
__device__ __forceinline__ void cell_fluxes2(const CoefPair& KP, const float* win, int aA, int aT, int aR, int d,
                                             f2 (&f)[5]) {
  constexpr int CELLS = PairShape<TX, TY>::CELLS;
  const f2 r = ld2(win + aR);
  const f2 H = ld2(win + aR + CELLS);
  const f2 u[3] = {ld2(win + aA), ld2(win + aA + CELLS), ld2(win + aA + 2 * CELLS)};
  const f2 ud = u[d];
  const f2 rud = r * ud;
  f[0] = rud;
#pragma unroll
  for (int i = 0; i < 3; ++i) f[1 + i] = i == d ? fma2(rud, ud, r * ld2(win + aT) * KP.inv_gamma) : rud * u[i];
  f[4] = H * ud;
}

// x-derivatives of a pair at cells q, q + 1 from the six cells q-2 .. q+3
// (three aligned 64-bit loads): first differences f[+1] - f[-1] and
// f[+2] - f[-2] of both points, or the sums for the second derivative.
struct XTaps {
  f2 A, B, C;   // cells (q-2, q-1), (q, q+1), (q+2, q+3)
  __device__ __forceinline__ f2 d1() const { return pk(B.y - A.y, C.x - B.x); }
  __device__ __forceinline__ f2 d2() const { return C - A; }
  __device__ __forceinline__ f2 s1() const { return pk(B.y + A.y, C.x + B.x); }
  __device__ __forceinline__ f2 s2() const { return C + A; }
};
__device__ __forceinline__ XTaps xtaps(const float* q) { return XTaps{ld2(q - 2), ld2(q), ld2(q + 2)}; }

// First-derivative coefficients (x 12) of the PE-local x-stencil of each
// point of a pair over the six-cell window starting at an even cell: central
// pairs start at x-2, the first two points of a PE row at x, the last two at
// x-4 (kinds of local_kind: 0 central, 1 first, 2 second, 3 second to last,
// 4 last point).
__device__ __forceinline__ void pair_xwindow(int kind0, float (&c0)[6], float (&c1)[6], int& start) {
#pragma unroll
  for (int j = 0; j < 6; ++j) c0[j] = c1[j] = 0.f;
  if (kind0 == 1) {          // points 0 and 1 of the PE: kinds 1 and 2 on x .. x+4
    const float a[5] = {-25, 48, -36, 16, -3}, b[5] = {-3, -10, 18, -6, 1};
#pragma unroll
    for (int j = 0; j < 5; ++j) { c0[j] = a[j]; c1[j] = b[j]; }
    start = 0;
  } else if (kind0 == 3) {   // last two points: kinds 3 and 4 on x-3 .. x+1
    const float a[5] = {-1, 6, -18, 10, 3}, b[5] = {3, -16, 36, -48, 25};
#pragma unroll
    for (int j = 0; j < 5; ++j) { c0[j + 1] = a[j]; c1[j + 1] = b[j]; }
    start = -4;
  } else {                   // central: x-2 .. x+2 and x-1 .. x+3
    const float a[5] = {1, -8, 0, 8, -1};
#pragma unroll
    for (int j = 0; j < 5; ++j) { c0[j] = a[j]; c1[j + 1] = a[j]; }
    start = -2;
  }
}

// One tile of the paired kernel: tile (bx, by) of TX x TY points, z chunk bz
// of ZC planes; blk is the tile's row in the statistics partials; smem is the
// dynamic shared memory (fused_smem_bytes<float>(TX, TY) bytes).  PLAIN
// compiles the step of the common configuration only -- an AB2 step that
// updates the state (no RK3 stage, no right-hand-side output), unforced, in
// the total-energy form with the power-law viscosity -- and leaves the code
// of the other configurations out of the kernel; the arithmetic of that
// configuration is the same in both instantiations.
template <int TX, int TY, bool PLAIN = false>
__device__ __forceinline__ void fused2_tile(const Geom& g, const Coef<float>& K, const CoefPair& KP,
                                            const StepArgs<float>& A, int ZC, int bx, int by, int bz, long long blk,
                                            unsigned char* smem) {
  const StepDyn<float> D = resolve_step(A);
  const bool eform = !PLAIN && K.eform, update = PLAIN || A.do_update, rk = !PLAIN && A.rk;
  using PS = PairShape<TX, TY>;
  using T_ = TileShape<TX, TY>;
  constexpr int CX = PS::CX, CELLS = PS::CELLS;
  float* win = reinterpret_cast<float*>(smem);
  FusedGeo F;
  F.x0 = bx * TX;
  F.y0 = by * TY;
  const int zs = bz * ZC;
  F.pe[0] = F.x0 / g.nl[0];
  F.pe[1] = F.y0 / g.nl[1];
  F.pe[2] = zs / g.nl[2];
  for (int d = 0; d < 3; ++d) F.base[d] = F.pe[d] * g.nl[d];
  const int tid = threadIdx.x;
  const int ty = tid / PS::TXH, txh = tid - ty * PS::TXH;
  const int x = F.x0 + 2 * txh, y = F.y0 + ty;                 // the pair is x, x + 1
  const int cell = (ty + 2) * CX + 2 + 2 * txh;                // window cell of the first point
  const long long N = g.npts;

  StatAcc<float> st;
  st.init();
  float wmax = 0.f, rmin = 3.0e38f, pmin = 3.0e38f;
  unsigned health = 0;

  const int li_x = x - F.base[0], li_y = y - F.base[1];
  const int kind_x = local_kind(g.pes[0], li_x, g.nl[0]);      // kind of the first point (the pair's is 1, 3 or 0)
  const int kind_y = local_kind(g.pes[1], li_y, g.nl[1]);
  float* FX = win + T_::OFF_FX;                                // [5][TY][CX]
  float* FY = win + T_::OFF_FY;                                // [5][CY][TX]
  float* XR = win + T_::OFF_XR;                                // [4][TY][CX]
  float* YC = win + T_::OFF_YC;                                // [4][CY][TX]
  const long long qsx = 4LL * g.pes[0] * g.plane[0], qsy = 4LL * g.pes[1] * g.plane[1];
  const long long qsz = 4LL * g.pes[2] * g.plane[2];

  // PE-local stencils of the mixed rule: x over a six-cell window with
  // per-point coefficients, y with the pair's common coefficients
  float lx0[6], lx1[6];
  int xstart;
  pair_xwindow(kind_x, lx0, lx1, xstart);
  f2 lcy[5];
  {
    float t0 = 1, t1 = -8, t2 = 0, t3 = 8, t4 = -1;      // kind 0: central
    if (kind_y == 1) { t0 = -25; t1 = 48; t2 = -36; t3 = 16; t4 = -3; }
    else if (kind_y == 2) { t0 = -3; t1 = -10; t2 = 18; t3 = -6; t4 = 1; }
    else if (kind_y == 3) { t0 = -1; t1 = 6; t2 = -18; t3 = 10; t4 = 3; }
    else if (kind_y == 4) { t0 = 3; t1 = -16; t2 = 36; t3 = -48; t4 = 25; }
    lcy[0] = bc(t0); lcy[1] = bc(t1); lcy[2] = bc(t2); lcy[3] = bc(t3); lcy[4] = bc(t4);
  }
  const int ax0 = ty * CX + 2 + 2 * txh + xstart;             // window start in an x-row array
  const int ay0 = (ty + 2 + local_first(kind_y)) * TX + 2 * txh;

  // z fluxes of this pair at window plane q = zp - zs + 4 (z ghosts beyond a PE z-face)
  auto zflux = [&](int zp, int q, f2 (&out)[5]) {
    if (F.beyond(g, 2, zp)) {
      const long long gi = checked((long long)(4 * F.pe[2] + F.ghost_slot(g, 2, zp)) * g.plane[2] +
                                       (long long)y * g.n[0] + x, qsz - 1, A.ds, CHK_GHOST);
#pragma unroll
      for (int e = 0; e < 5; ++e) out[e] = ld2(A.GH[2] + e * qsz + gi);
    } else {
      cell_fluxes2<TX, TY>(KP, win, slot_A<TX, TY>(q) + cell, slot_T<TX, TY>(q) + cell, slot_R<TX, TY>(q) + cell, 2,
                           out);
    }
  };

  for (int q = 0; q < 8; ++q) {
    PlaneRaw2<TX, TY> P;
    fetch_plane2<TX, TY>(g, A, D.U, F, zs - 4 + q, P);
    store_plane2<TX, TY, PLAIN>(K, KP, P, win, slot_A<TX, TY>(q), slot_T<TX, TY>(q), slot_R<TX, TY>(q));
  }
  PlaneRaw2<TX, TY> pf;                                       // plane z + 4, fetched one iteration ahead
  fetch_plane2<TX, TY>(g, A, D.U, F, zs + 4, pf);

  for (int z = zs; z < zs + ZC; ++z) {
    const int q = z - zs + 4;
    store_plane2<TX, TY, PLAIN>(K, KP, pf, win, slot_A<TX, TY>(q + 4), slot_T<TX, TY>(q + 4), slot_R<TX, TY>(q + 4));
    __syncthreads();
    if (z + 1 < zs + ZC) fetch_plane2<TX, TY>(g, A, D.U, F, z + 5, pf);
    const long long idx = checked(((long long)z * g.n[1] + y) * g.n[0] + x, N - 1, A.ds, CHK_STATE);
    const f2 m[3] = {ld2(D.U + N + idx), ld2(D.U + 2 * N + idx), ld2(D.U + 3 * N + idx)};
    const f2 Ecur = ld2(D.U + 4 * N + idx);
    f2 Rp[5], Lp[5];
    const bool ldrp = needs_rprev(A, D), ldlo = update && D.Ulo;
#pragma unroll
    for (int v = 0; v < 5; ++v) Rp[v] = ldrp ? ld2(A.Rprev + v * N + idx) : bc(0.f);
    // the compensated form's low words of U^n, loaded with R^{n-1}
#pragma unroll
    for (int v = 0; v < 5; ++v) Lp[v] = ldlo ? ld2(D.Ulo + v * N + idx) : bc(0.f);

    // ---- per-plane flux arrays and AT derivative arrays, on cell pairs
    {
      const int bA = slot_A<TX, TY>(q), bT = slot_T<TX, TY>(q), bR = slot_R<TX, TY>(q);
      const int bAm1 = slot_A<TX, TY>(q - 1), bAp1 = slot_A<TX, TY>(q + 1);
      const int bAm2 = slot_A<TX, TY>(q - 2), bAp2 = slot_A<TX, TY>(q + 2);
      auto ddz = [&](int f, int cw) {
        const int o = f * CELLS + cw;
        return fma2(KP.c1[2], ld2(win + bAp1 + o) - ld2(win + bAm1 + o),
                    KP.c2[2] * (ld2(win + bAp2 + o) - ld2(win + bAm2 + o)));
      };
      auto ddy = [&](const float* p) {
        return fma2(KP.c1[1], ld2(p + CX) - ld2(p - CX), KP.c2[1] * (ld2(p + 2 * CX) - ld2(p - 2 * CX)));
      };
      auto ddx = [&](const float* p) {
        const XTaps t = xtaps(p);
        return fma2(KP.c1[0], t.d1(), KP.c2[0] * t.d2());
      };
      constexpr int XPR = CX / 2, XP = TY * XPR;        // x-row pairs
      constexpr int YPR = TX / 2, YP = (TY + 4) * YPR;  // y-column pairs
      // one loop over both kinds of pair, so the passes spread evenly over the
      // threads; the y-column pairs come first: their count, (TY + 4) TX / 2,
      // is a multiple of 32 for every tile, so no warp holds pairs of both
      // kinds.  The x-row pairs follow, the TY TX / 2 pairs of the tile's own
      // columns (again whole warps) before the 2 TY x-halo pairs, so that the
      // halo pairs' ghost loads do not diverge inside the warps that compute
      // fluxes.
      static_assert(YP % 32 == 0 && (TY * (TX / 2)) % 32 == 0, "pair groups fill whole warps");
      constexpr int XPI = TY * (TX / 2);                // x-row pairs of the tile's own columns
      for (int pi = tid; pi < XP + YP; pi += PS::NT) {
        if (pi >= YP) {
        const int p = pi - YP;
        int r, cxw;
        if (p < XPI) {
          r = p / (TX / 2);
          cxw = 2 + 2 * (p - r * (TX / 2));
        } else {
          r = (p - XPI) >> 1;
          cxw = ((p - XPI) & 1) ? CX - 2 : 0;
        }
        const int c = r * CX + cxw;
        const int xg = F.x0 - 2 + cxw, yg = F.y0 + r;
        const int cw = (r + 2) * CX + cxw;
        if (F.beyond(g, 0, xg)) {
          const long long g0 = checked((long long)(4 * F.pe[0] + F.ghost_slot(g, 0, xg)) * g.plane[0] +
                                           (long long)z * g.n[1] + yg, qsx - g.plane[0], A.ds, CHK_GHOST);
          const long long g1 = g0 + g.plane[0];
#pragma unroll
          for (int e = 0; e < 5; ++e) st2(FX + e * TY * CX + c, pk(A.GH[0][e * qsx + g0], A.GH[0][e * qsx + g1]));
        } else {
          f2 f[5];
          cell_fluxes2<TX, TY>(KP, win, bA + cw, bT + cw, bR + cw, 0, f);
#pragma unroll
          for (int e = 0; e < 5; ++e) st2(FX + e * TY * CX + c, f[e]);
        }
        // (pairs beyond the x-face are never read by the PE-local x-stencils)
        st2(XR + XR_VY * TY * CX + c, ddy(win + bA + CELLS + cw));
        st2(XR + XR_UY * TY * CX + c, ddy(win + bA + cw));
        st2(XR + XR_WZ * TY * CX + c, ddz(2, cw));
        st2(XR + XR_UZ * TY * CX + c, ddz(0, cw));
        } else {
        const int py = pi;
        const int r = py / YPR, cxl = 2 * (py - r * YPR);
        const int c = r * TX + cxl;
        const int xg = F.x0 + cxl, yg = F.y0 - 2 + r;
        const int cw = r * CX + cxl + 2;
        if (F.beyond(g, 1, yg)) {
          const long long gi = checked((long long)(4 * F.pe[1] + F.ghost_slot(g, 1, yg)) * g.plane[1] +
                                           (long long)z * g.n[0] + xg, qsy - 1, A.ds, CHK_GHOST);
#pragma unroll
          for (int e = 0; e < 5; ++e) st2(FY + e * (TY + 4) * TX + c, ld2(A.GH[1] + e * qsy + gi));
        } else {
          f2 f[5];
          cell_fluxes2<TX, TY>(KP, win, bA + cw, bT + cw, bR + cw, 1, f);
#pragma unroll
          for (int e = 0; e < 5; ++e) st2(FY + e * (TY + 4) * TX + c, f[e]);
        }
        st2(YC + YC_VX * (TY + 4) * TX + c, ddx(win + bA + CELLS + cw));
        st2(YC + YC_UX * (TY + 4) * TX + c, ddx(win + bA + cw));
        st2(YC + YC_WZ * (TY + 4) * TX + c, ddz(2, cw));
        st2(YC + YC_VZ * (TY + 4) * TX + c, ddz(1, cw));
        }
      }
    }
    __syncthreads();

    int pA[kWinPlanes], pT[5];
#pragma unroll
    for (int k = 0; k < kWinPlanes; ++k) pA[k] = slot_A<TX, TY>(q - 4 + k) + cell;
#pragma unroll
    for (int k = 0; k < 5; ++k) pT[k] = slot_T<TX, TY>(q - 2 + k) + cell;
    const int pR = slot_R<TX, TY>(q) + cell;
    const int li_z = z - F.base[2];
    const int kind_z = local_kind(g.pes[2], li_z, g.nl[2]);
    // field f (0 u, 1 v, 2 w, 3 T) of the pair at plane offset dz (|dz| <= 4 for u, v, w; <= 2 for T)
    auto fp = [&](int f, int dz) -> const float* {
      return f < 3 ? win + pA[4 + dz] + f * CELLS : win + pT[2 + dz];
    };

    // ---- inviscid flux divergence -sum_d D_d F_d
    f2 dz1[5], dz2[5];
    {
      f2 fa[5], fb[5];
      zflux(z + 1, q + 1, fa);
      zflux(z - 1, q - 1, fb);
#pragma unroll
      for (int e = 0; e < 5; ++e) dz1[e] = fa[e] - fb[e];
      zflux(z + 2, q + 2, fa);
      zflux(z - 2, q - 2, fb);
#pragma unroll
      for (int e = 0; e < 5; ++e) dz2[e] = fa[e] - fb[e];
    }
    f2 R[5];
#pragma unroll
    for (int e = 0; e < 5; ++e) {
      const XTaps tx = xtaps(FX + e * TY * CX + ty * CX + 2 + 2 * txh);
      const float* fy = FY + e * (TY + 4) * TX + (ty + 2) * TX + 2 * txh;
      f2 acc = KP.nc1[0] * tx.d1();
      acc = fma2(KP.nc2[0], tx.d2(), acc);
      acc = fma2(KP.nc1[1], ld2(fy + TX) - ld2(fy - TX), acc);
      acc = fma2(KP.nc2[1], ld2(fy + 2 * TX) - ld2(fy - 2 * TX), acc);
      acc = fma2(KP.nc1[2], dz1[e], acc);
      R[e] = fma2(KP.nc2[2], dz2[e], acc);
    }

    // ---- second derivatives of u, v, w, T; first derivatives at the points
    f2 lap[4], d2diag[3], Ag[3][3], dT[3];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const float* c0 = fp(f, 0);
      const XTaps tx = xtaps(c0);
      const f2 f0 = tx.B;
      f2 off[3], d1[3];
      off[0] = fma2(KP.a1[0], tx.s1(), KP.a2[0] * tx.s2());
      d1[0] = fma2(KP.c1[0], tx.d1(), KP.c2[0] * tx.d2());
      {
        const f2 ym1 = ld2(c0 - CX), yp1 = ld2(c0 + CX), ym2 = ld2(c0 - 2 * CX), yp2 = ld2(c0 + 2 * CX);
        off[1] = fma2(KP.a1[1], yp1 + ym1, KP.a2[1] * (yp2 + ym2));
        d1[1] = fma2(KP.c1[1], yp1 - ym1, KP.c2[1] * (yp2 - ym2));
      }
      {
        const f2 zm1 = ld2(fp(f, -1)), zp1 = ld2(fp(f, 1)), zm2 = ld2(fp(f, -2)), zp2 = ld2(fp(f, 2));
        off[2] = fma2(KP.a1[2], zp1 + zm1, KP.a2[2] * (zp2 + zm2));
        d1[2] = fma2(KP.c1[2], zp1 - zm1, KP.c2[2] * (zp2 - zm2));
      }
      lap[f] = fma2(KP.a0sum, f0, off[0] + off[1] + off[2]);
      if (f < 3) {
        d2diag[f] = fma2(KP.a0[f], f0, off[f]);
#pragma unroll
        for (int d = 0; d < 3; ++d) Ag[f][d] = d1[d];
      } else {
#pragma unroll
        for (int d = 0; d < 3; ++d) dT[d] = d1[d];
      }
    }

    // ---- d theta/dx_i with the mixed terms by the three-step rule (Sec. 2.1)
    f2 gth[3];
    {
      constexpr int sxr = TY * CX, syc = (TY + 4) * TX;
      const bool bx_ = kind_x != 0, by_ = kind_y != 0, bz_ = kind_z != 0;
      const bool bxy = bx_ || by_, bxz = bx_ || bz_, byz = by_ || bz_;
      auto mix = [&](f2 pa, f2 pb, bool bnd) { return bnd ? bc(0.5f) * (pa + pb) : pa; };
      // x-stencil of an x-row array over the pair's six-cell window
      auto tx_ = [&](int fld) {
        const float* p = XR + fld * sxr + ax0;
        const f2 w0 = ld2(p), w1 = ld2(p + 2), w2 = ld2(p + 4);
        const float w[6] = {w0.x, w0.y, w1.x, w1.y, w2.x, w2.y};
        float a = 0.f, b = 0.f;
#pragma unroll
        for (int j = 0; j < 6; ++j) {
          a = fmaf(lx0[j], w[j], a);
          b = fmaf(lx1[j], w[j], b);
        }
        return pk(a, b);
      };
      auto ty_ = [&](int fld) {
        const float* p = YC + fld * syc + ay0;
        f2 acc = lcy[0] * ld2(p);
#pragma unroll
        for (int i = 1; i < 5; ++i) acc = fma2(lcy[i], ld2(p + i * TX), acc);
        return acc;
      };
      // 12 dz times the PE-local derivative along z (CTA-uniform kind) of the
      // AT derivative of field f along `in` (0: x, 1: y)
      auto zl = [&](int f, int in) {
        auto dv = [&](int o) {
          const float* c0 = fp(f, o);
          if (in == 1) return fma2(KP.c1[1], ld2(c0 + CX) - ld2(c0 - CX), KP.c2[1] * (ld2(c0 + 2 * CX) - ld2(c0 - 2 * CX)));
          const XTaps t = xtaps(c0);
          return fma2(KP.c1[0], t.d1(), KP.c2[0] * t.d2());
        };
        constexpr float c[5][5] = {{1, -8, 0, 8, -1}, {-25, 48, -36, 16, -3}, {-3, -10, 18, -6, 1},
                                   {-1, 6, -18, 10, 3}, {3, -16, 36, -48, 25}};
        auto taps = [&](auto KIND) {
          constexpr int k = decltype(KIND)::value;
          if constexpr (k == 0) {
            return fma2(bc(8.f), dv(1) - dv(-1), dv(-2) - dv(2));
          } else {
            f2 acc = bc(c[k][0]) * dv(local_first(k));
#pragma unroll
            for (int i = 1; i < 5; ++i) acc = fma2(bc(c[k][i]), dv(local_first(k) + i), acc);
            return acc;
          }
        };
        switch (kind_z) {
          case 0: return taps(std::integral_constant<int, 0>{});
          case 1: return taps(std::integral_constant<int, 1>{});
          case 2: return taps(std::integral_constant<int, 2>{});
          case 3: return taps(std::integral_constant<int, 3>{});
          default: return taps(std::integral_constant<int, 4>{});
        }
      };
      const f2 m_xy = mix(KP.hloc[0] * tx_(XR_VY), KP.hloc[1] * ty_(YC_VX), bxy);
      const f2 m_yx = mix(KP.hloc[1] * ty_(YC_UX), KP.hloc[0] * tx_(XR_UY), bxy);
      const f2 pa_xz = KP.hloc[0] * tx_(XR_WZ);
      const f2 pb_xz = __any_sync(__activemask(), bxz) ? KP.hloc[2] * zl(2, 0) : bc(0.f);
      const f2 pa_zx = KP.hloc[2] * zl(0, 0);
      const f2 pb_zx = KP.hloc[0] * tx_(XR_UZ);
      const f2 pa_yz = KP.hloc[1] * ty_(YC_WZ);
      const f2 pb_yz = __any_sync(__activemask(), byz) ? KP.hloc[2] * zl(2, 1) : bc(0.f);
      const f2 pa_zy = KP.hloc[2] * zl(1, 1);
      const f2 pb_zy = KP.hloc[1] * ty_(YC_VZ);
      gth[0] = d2diag[0] + m_xy + mix(pa_xz, pb_xz, bxz);
      gth[1] = d2diag[1] + m_yx + mix(pa_yz, pb_yz, byz);
      gth[2] = d2diag[2] + mix(pa_zx, pb_zx, bxz) + mix(pa_zy, pb_zy, byz);
    }

    // ---- point values and assembly (Sec. 2)
    const f2 r = ld2(win + pR);
    const f2 vel[3] = {ld2(win + pA[4]), ld2(win + pA[4] + CELLS), ld2(win + pA[4] + 2 * CELLS)};
    const f2 T = ld2(win + pT[2]);
    const f2 p = eform ? KP.gm1 * Ecur
                         : KP.gm1 * fma2(bc(-0.5f), fma2(m[0], vel[0], fma2(m[1], vel[1], m[2] * vel[2])), Ecur);
    const f2 theta = Ag[0][0] + Ag[1][1] + Ag[2][2];
    f2 mu, dmudT;
    {
      float mu0_, mu1_, d0_, d1_;
      if constexpr (PLAIN) {
        viscosity_power32(K, T.x, mu0_, d0_);
        viscosity_power32(K, T.y, mu1_, d1_);
      } else {
        viscosity(K, T.x, mu0_, d0_);
        viscosity(K, T.y, mu1_, d1_);
      }
      mu = pk(mu0_, mu1_);
      dmudT = pk(d0_, d1_);
    }
    const f2 kappa = mu * KP.cp_over_pr;
    f2 dmu[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) dmu[j] = dmudT * dT[j];
    f2 sm[3][3];
    const f2 th23 = bc(2.0f / 3.0f) * theta;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) sm[i][j] = i == j ? fma2(bc(2.f), Ag[i][i], bc(0.f) - th23) : Ag[i][j] + Ag[j][i];

    f2 fo[3] = {bc(0.f), bc(0.f), bc(0.f)};
    if (!PLAIN && A.fB) {
      const long long lines = (long long)g.n[2] * g.n[1];
      const long long ln = (long long)z * g.n[1] + y;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        f2 acc = bc(0.f);
        for (int kx = 0; kx <= A.fK; ++kx) {
          const float2 b = A.fB[((long long)kx * 3 + c) * lines + ln];
          const float4 e = *reinterpret_cast<const float4*>(A.fX + (long long)kx * g.n[0] + x);   // x, x + 1
          // Re(b e^{i kx x}) = b.x cos - b.y sin, for both points
          acc = fma2(bc(b.x), pk(e.x, e.z), fma2(bc(-b.y), pk(e.y, e.w), acc));
        }
        fo[c] = acc;
      }
    }

    f2 sS = sm[0][0] * Ag[0][0];
    sS = fma2(sm[1][1], Ag[1][1], sS);
    sS = fma2(sm[2][2], Ag[2][2], sS);
    sS = fma2(sm[0][1], sm[0][1], sS);
    sS = fma2(sm[0][2], sm[0][2], sS);
    sS = fma2(sm[1][2], sm[1][2], sS);
    const f2 sigS = mu * sS;
    f2 work = bc(0.f);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      f2 V = mu * fma2(gth[i], bc(1.0f / 3.0f), lap[i]);
#pragma unroll
      for (int j = 0; j < 3; ++j) V = fma2(dmu[j], sm[i][j], V);
      R[1 + i] = R[1 + i] + (PLAIN ? V : fma2(r, fo[i], V));   // (no forcing in PLAIN)
      work = fma2(vel[i], V, work);
    }
    const f2 heat = fma2(KP.cp_over_pr, fma2(dmu[0], dT[0], fma2(dmu[1], dT[1], dmu[2] * dT[2])), kappa * lap[3]);
    if (eform) R[4] = R[4] + fma2(bc(0.f) - p, theta, sigS + heat);
    else if (PLAIN) R[4] = R[4] + (sigS + work + heat);
    else R[4] = R[4] + fma2(r, fma2(fo[0], vel[0], fma2(fo[1], vel[1], fo[2] * vel[2])), sigS + work + heat);

    if (nonpositive(r.x) || nonpositive(r.y)) health |= H_RHO;
    if (nonpositive(p.x) || nonpositive(p.y)) health |= H_P;
    // (a step that updates checks U^{n+1}, which is not finite where R is not)
    if (!update) {
#pragma unroll
      for (int v = 0; v < 5; ++v)
        if (nonfinite(R[v].x) || nonfinite(R[v].y)) health |= H_NONFINITE;
    }

    if (update) {
      const f2 Uo[5] = {r, m[0], m[1], m[2], Ecur};
      f2 un[5], unlo[5];
      const f2 scale = rk ? bc(1.f) : KP.dt;
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        f2 inc, kept;
        if (rk) {
          kept = fma2(bc(A.rkA), Rp[v], KP.dt * R[v]);   // stage register dU
          inc = bc(A.rkB) * kept;
        } else {
          inc = D.first ? R[v] : fma2(bc(1.5f), R[v], bc(-0.5f) * Rp[v]);
          kept = R[v];
        }
        if (D.Ulo) {
          // TwoSum(U_hi, dt inc) into the low word, then renormalise
          const f2 dlt = scale * inc;
          const f2 s = Uo[v] + dlt;
          const f2 bp = s - Uo[v];
          const f2 e = (Uo[v] - (s - bp)) + (dlt - bp);
          const f2 lo = Lp[v] + e;
          const f2 hi = s + lo;
          unlo[v] = lo - (hi - s);
          un[v] = hi;
          st2(D.Ulo_next + v * N + idx, unlo[v]);
        } else {
          un[v] = fma2(scale, inc, Uo[v]);
          unlo[v] = bc(0.f);
        }
        st2(D.Unext + v * N + idx, un[v]);
        st2(A.Rprev + v * N + idx, kept);
        if (nonfinite(un[v].x) || nonfinite(un[v].y)) health |= H_NONFINITE;
      }
      // (the ring slabs of level n+1 are written by the next step's ghost kernel)
      if (A.xst && g.pes[0] > 1 && (li_x < 2 || li_x >= g.nl[0] - 2)) {
        // the pair is x-face slabs t and t + 1 of its PE
        const int t = li_x < 2 ? li_x : li_x - g.nl[0] + 4;
        const long long pv = 4LL * g.pes[0] * g.plane[0];
        float* o = A.xst + checked((4LL * F.pe[0] + t) * g.plane[0] + (long long)z * g.n[1] + y,
                                   4LL * g.pes[0] * g.plane[0] - g.plane[0], A.ds, CHK_STAGE);
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          o[v * pv] = un[v].x;
          o[v * pv + g.plane[0]] = un[v].y;
          if (A.xst_half) {
            o[A.xst_half + v * pv] = unlo[v].x;
            o[A.xst_half + v * pv + g.plane[0]] = unlo[v].y;
          }
        }
      }
    } else if (!PLAIN && A.Rout) {
#pragma unroll
      for (int v = 0; v < 5; ++v)
        *reinterpret_cast<double2*>(A.Rout + v * N + idx) = make_double2(f2d_bits(R[v].x), f2d_bits(R[v].y));
    }

    if (A.do_stats) {
      const f2 uu = fma2(vel[0], vel[0], fma2(vel[1], vel[1], vel[2] * vel[2]));
      const f2 c = pk(sqrtf(T.x), sqrtf(T.y));
      auto add = [&](int i, f2 v) { st.add(i, v.x + v.y); };
      add(ST_RHO, r);
      add(ST_M0, m[0]);
      add(ST_M1, m[1]);
      add(ST_M2, m[2]);
      add(ST_E, Ecur);
      add(ST_KE, bc(0.5f) * r * uu);
      add(ST_SIGS, sigS);
      const f2 a0 = Ag[0][0], a1 = Ag[1][1], a2 = Ag[2][2];
      const f2 q0 = a0 * a0, q1 = a1 * a1, q2 = a2 * a2;
      add(ST_G2, q0 + q1 + q2);
      add(ST_G3, fma2(q0, a0, fma2(q1, a1, q2 * a2)));
      add(ST_G4, fma2(q0, q0, fma2(q1, q1, q2 * q2)));
      const f2 o0 = Ag[2][1] - Ag[1][2], o1 = Ag[0][2] - Ag[2][0], o2 = Ag[1][0] - Ag[0][1];
      add(ST_ENST, fma2(o0, o0, fma2(o1, o1, o2 * o2)));
      add(ST_PTHETA, p * theta);
      if (!PLAIN) add(ST_FPOW, r * fma2(fo[0], vel[0], fma2(fo[1], vel[1], fo[2] * vel[2])));
      add(ST_U2, uu);
      add(ST_C, c);
      wmax = fmaxf(wmax, fmaxf(fmaxf(fabsf(vel[0].x), fabsf(vel[1].x)), fabsf(vel[2].x)) + c.x);
      wmax = fmaxf(wmax, fmaxf(fmaxf(fabsf(vel[0].y), fabsf(vel[1].y)), fabsf(vel[2].y)) + c.y);
      rmin = fminf(rmin, fminf(r.x, r.y));
      pmin = fminf(pmin, fminf(p.x, p.y));
    }
    __syncthreads();
  }
  long long kwave = LLONG_MIN, krho = LLONG_MAX, kp = LLONG_MAX;
  if (A.do_stats) {
    kwave = okey(wmax);
    krho = okey(rmin);
    kp = okey(pmin);
  }
  block_reduce<float, (PS::NT > 256 ? 512 : (PS::NT > 128 ? 256 : 128))>(
      st.s, kwave, krho, kp, health, A.do_stats != 0, A.partial, A.words, reinterpret_cast<double*>(smem), st.c, blk);
}

template <int TX, int TY, bool PLAIN>
__global__ void __launch_bounds__(TX * TY / 2, (TX * TY / 2 <= 128) ? 2 : 1)
    k_fused2(Geom g, Coef<float> K, CoefPair KP, StepArgs<float> A0, int ZC) {
  extern __shared__ __align__(16) unsigned char fused_smem[];
  const long long blk = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  fused2_tile<TX, TY, PLAIN>(g, K, KP, A0, ZC, blockIdx.x, blockIdx.y, blockIdx.z, blk, fused_smem);
}

}  // namespace atdns
