// AT-DNS step kernels, templated on the scalar type S (double for the FP64
// form, float for the FP32-bulk forms).  The stencils, the AT extrapolation
// and the update run in S; the slab ring of past levels is FP64 in every form
// (the FP32 forms write and read it with integer instructions); the
// statistics are summed in FP64 across points in a fixed order (FP32 forms:
// compensated FP32 sums within a block first).
//
// One RHS evaluation (Sec. 2) is four launches:
//   k_prim   per point: u, v, w, T and the 12 non-trivial inviscid fluxes;
//   k_ghost  per PE-face ghost point (M layers each side, Sec. 3; M = 2 for
//            the 4th-order scheme, 3 for the 6th-order one): the 9
//            differentiated quantities of that direction at level n (k = 0) or
//            extrapolated from levels n-k .. n-k-M of the slab ring with the
//            Table B weights (Appendix B);
//   k_grad   per point: AT first derivatives du_i/dx_j and dT/dx_j;
//   k_main   per point: inviscid flux divergence, second derivatives, mixed
//            derivatives by the three-step rule (Sec. 2.1), viscous / heat /
//            forcing assembly, AB2 update (Eq. (time_ab)), ring write of the
//            new PE-boundary slabs and the block reductions.
//
// Floating-point work is kept off the FP64 pipe in the FP32 form (constants
// come converted from the host, sign tests and min/max use bit patterns).
#pragma once
#include <climits>
#include "common.cuh"

namespace atdns {

// ---------------------------------------------------------------------------
template <typename S>
__global__ void __launch_bounds__(256) k_prim(Geom g, Coef<S> K, const S* __restrict__ U0, const S* __restrict__ U1,
                                              const DevState* __restrict__ ds, S* __restrict__ PQ) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= g.npts) return;
  const S* __restrict__ U = (ds && ds->cur) ? U1 : U0;
  const long long N = g.npts;
  const S r = U[idx], m0 = U[N + idx], m1 = U[2 * N + idx], m2 = U[3 * N + idx], E = U[4 * N + idx];
  const S inv = S(1) / r;
  const S u = m0 * inv, v = m1 * inv, w = m2 * inv;
  const S p = pressure(K, m0, m1, m2, u, v, w, E);
  const S T = K.gamma * p * inv;
  const S H = K.eform ? E : E + p;   // fifth flux = H u_d
  PQ[0 * N + idx] = u;
  PQ[1 * N + idx] = v;
  PQ[2 * N + idx] = w;
  PQ[3 * N + idx] = T;
  // flux of direction d, components e = 1..4: rho u_i u_d + p delta_id, (E+p) u_d
  PQ[4 * N + idx] = fma(m0, u, p);
  PQ[5 * N + idx] = m1 * u;
  PQ[6 * N + idx] = m2 * u;
  PQ[7 * N + idx] = H * u;
  PQ[8 * N + idx] = m0 * v;
  PQ[9 * N + idx] = fma(m1, v, p);
  PQ[10 * N + idx] = m2 * v;
  PQ[11 * N + idx] = H * v;
  PQ[12 * N + idx] = m0 * w;
  PQ[13 * N + idx] = m1 * w;
  PQ[14 * N + idx] = fma(m2, w, p);
  PQ[15 * N + idx] = H * w;
}

// a, b or c for direction d = 0, 1, 2 (selects: no dynamically indexed
// arrays, which the compiler would place in local memory).
template <typename S>
__device__ __forceinline__ S sel3(int d, S a, S b, S c) { return d == 0 ? a : (d == 1 ? b : c); }

// The 9 quantities of direction d from one level of U (same arithmetic as k_prim).
template <typename S>
__device__ __forceinline__ void ghost_quantities(const Coef<S>& K, int d, const S* Uv, S* q) {
  const S r = Uv[0], inv = S(1) / r;
  const S vel[3] = {Uv[1] * inv, Uv[2] * inv, Uv[3] * inv};
  const S p = pressure(K, Uv[1], Uv[2], Uv[3], vel[0], vel[1], vel[2], Uv[4]);
  const S T = K.gamma * p * inv;
  const S ud = sel3(d, vel[0], vel[1], vel[2]);
  q[0] = sel3(d, Uv[1], Uv[2], Uv[3]);
  q[1] = fma(Uv[1], ud, d == 0 ? p : S(0));
  q[2] = fma(Uv[2], ud, d == 1 ? p : S(0));
  q[3] = fma(Uv[3], ud, d == 2 ? p : S(0));
  q[4] = (K.eform ? Uv[4] : Uv[4] + p) * ud;
  q[5] = vel[0];
  q[6] = vel[1];
  q[7] = vel[2];
  q[8] = T;
}

// FP32 forms: the AT ghost value sum_l w_l q(U^{n-k-l}) from FP64 levels.
// With B = level n-k truncated to FP32 and sum_l w_l = 1 (Table B), it is
// q(B) + sum_l w_l [q(U_l) - q(B)]; each difference is formed from
// dU_l = U_l - B (exact in FP32 up to rounding of the difference itself) by
// the identities
//   d(a b) = da b + (a + da) db,          du_i = (dm_i - u_i drho) / (rho + drho),
//   dp = (gamma-1) (dE - d(m.u)/2),       dT = (gamma dp - T drho) / (rho + drho),
// so the rounding error stays relative to q (not amplified by Table B's
// weights, sum_l |w_l| = 17 at k = 2 and 111 at k = 3 for the 6th order) and
// to the differences, which are small.  Integer instructions split the FP64
// values (no FP64 arithmetic in the FP32 kernels).
struct GhostBase {
  float r, m0, m1, m2, E;    // B, level n-k truncated to FP32
  float u0, u1, u2, p, T, H; // its primitives and the fifth flux's factor
};

__device__ __forceinline__ GhostBase ghost_base(const Coef<float>& K, float r, float m0, float m1, float m2, float E) {
  GhostBase B;
  B.r = r;
  B.m0 = m0;
  B.m1 = m1;
  B.m2 = m2;
  B.E = E;
  const float inv = rcp_rn(r);
  B.u0 = m0 * inv;
  B.u1 = m1 * inv;
  B.u2 = m2 * inv;
  B.p = pressure(K, m0, m1, m2, B.u0, B.u1, B.u2, E);
  B.T = K.gamma * B.p * inv;
  B.H = K.eform ? E : E + B.p;
  return B;
}

// acc += w (q(B + dU) - q(B)) for the 9 quantities of direction d.
__device__ __forceinline__ void ghost_delta_f32(const Coef<float>& K, int d, const GhostBase& B, float dr, float dm0,
                                                float dm1, float dm2, float dE, float w, float* acc) {
  const float inv2 = rcp_rn(B.r + dr);
  const float du0 = fmaf(-B.u0, dr, dm0) * inv2;
  const float du1 = fmaf(-B.u1, dr, dm1) * inv2;
  const float du2 = fmaf(-B.u2, dr, dm2) * inv2;
  const float n0 = B.m0 + dm0, n1 = B.m1 + dm1, n2 = B.m2 + dm2;   // m + dm
  const float dmu = fmaf(dm0, B.u0, fmaf(n0, du0, fmaf(dm1, B.u1, fmaf(n1, du1, fmaf(dm2, B.u2, n2 * du2)))));
  const float dp = K.eform ? K.gm1 * dE : K.gm1 * fmaf(-0.5f, dmu, dE);
  const float dH = K.eform ? dE : dE + dp;
  const float ud = sel3(d, B.u0, B.u1, B.u2), dud = sel3(d, du0, du1, du2);
  acc[0] = fmaf(w, sel3(d, dm0, dm1, dm2), acc[0]);
  acc[1] = fmaf(w, fmaf(dm0, ud, n0 * dud) + (d == 0 ? dp : 0.f), acc[1]);
  acc[2] = fmaf(w, fmaf(dm1, ud, n1 * dud) + (d == 1 ? dp : 0.f), acc[2]);
  acc[3] = fmaf(w, fmaf(dm2, ud, n2 * dud) + (d == 2 ? dp : 0.f), acc[3]);
  acc[4] = fmaf(w, fmaf(dH, ud, (B.H + dH) * dud), acc[4]);
  acc[5] = fmaf(w, du0, acc[5]);
  acc[6] = fmaf(w, du1, acc[6]);
  acc[7] = fmaf(w, du2, acc[7]);
  acc[8] = fmaf(w, fmaf(K.gamma, dp, -B.T * dr) * inv2, acc[8]);
}

// ---------------------------------------------------------------------------
// AT ghost assembly.  Ghost slot s of PE column p_d along d (2M slots): s < M
// is the local coordinate s - M (left face, face 2d), s >= M is nl + s - M
// (right face, face 2d+1).  Ring slab index sp = 2M p + t with t < M for
// local t and t >= M for local nl - 2M + t.
// One ghost point j (counted over the three directions: cnt0, cnt1, cnt2
// points) of the step at level n; delay(p, face) gives the delay of face
// `face` of PE p at this step.
template <typename S, int M, typename Delay>
__device__ __forceinline__ void ghost_point(const Geom& g, const Coef<S>& K, const S* __restrict__ U0,
                                            const S* __restrict__ U1, const S* __restrict__ Ulo0,
                                            const S* __restrict__ Ulo1, const DevState* __restrict__ ds,
                                            const S* __restrict__ PQ, S* GH0, S* GH1, S* GH2,
                                            double* __restrict__ ring0, double* __restrict__ ring1,
                                            double* __restrict__ ring2, const S* __restrict__ xst,
                                            long long xst_half, Delay delay, long long n, long long cnt0,
                                            long long cnt1, long long cnt2, long long j) {
  const S* __restrict__ U = (ds && ds->cur) ? U1 : U0;
  const S* __restrict__ Ulo = (ds && ds->cur) ? Ulo1 : Ulo0;   // compensated form: low words (else null)
  if (ds) n = ds->n;
  int d;
  if (j < cnt0) d = 0;
  else if ((j -= cnt0) < cnt1) d = 1;
  else if ((j -= cnt1) < cnt2) d = 2;
  else return;
  S* GH = d == 0 ? GH0 : (d == 1 ? GH1 : GH2);
  double* ring = d == 0 ? ring0 : (d == 1 ? ring1 : ring2);
  // j < 2M P_d plane_d < npts < 2^31 (grids hold fewer than 2^31 points), so
  // the index arithmetic below runs in 32 bits (no 64-bit division)
  const unsigned plane = (unsigned)g.plane[d];
  constexpr int NS = 2 * M;
  const unsigned ju = (unsigned)j;
  const int gi = (int)(ju / plane);
  const unsigned pl = ju - (unsigned)gi * plane;
  const int ped = gi / NS, slot = gi - ped * NS;
  const int P = g.pes[d], nl = g.nl[d], nd = g.n[d];
  int c[3];
  {
    const unsigned row = (unsigned)(d == 0 ? g.n[1] : g.n[0]);   // fastest extent of the face plane
    const int hi = (int)(pl / row), lo = (int)(pl - (unsigned)hi * row);
    if (d == 0) { c[2] = hi; c[1] = lo; }
    else if (d == 1) { c[2] = hi; c[0] = lo; }
    else { c[1] = hi; c[0] = lo; }
  }
  int cd = ped * nl + (slot < M ? slot - M : nl + slot - M);
  cd = cd < 0 ? cd + nd : (cd >= nd ? cd - nd : cd);
  c[d] = ped * nl;   // any coordinate inside the receiving PE
  const int p = pe_number(g, c[0], c[1], c[2]);
  const int face = 2 * d + (slot >= M ? 1 : 0);
  const int k = delay(p, face);
  const long long qstride = (long long)NS * P * plane;   // points of the direction's slabs
  S* out = GH + checked((long long)gi * plane + pl, qstride, ds, CHK_GHOST);
  // the source point (in the neighbouring PE) and its slab of the ring
  c[d] = cd;
  const long long N = g.npts;
  const long long src = checked(((long long)c[2] * g.n[1] + c[1]) * g.n[0] + c[0], N, ds, CHK_STATE);
  const int nbr = slot < M ? (ped - 1 + P) % P : (ped + 1) % P;
  const int sp = NS * nbr + (slot < M ? slot + M : slot - M);
  const long long spp = checked((long long)sp * plane + pl, qstride, ds, CHK_RING);   // slab point
  const int nm = ring_slot(g, n);
  // Level n of the source point into its ring slot: every slab point of the
  // ring is the source of exactly one ghost slot, and no ghost reads the slot
  // of level n from the ring (delay 0 reads the state), so this kernel keeps
  // the ring current for the later steps that read level n with a delay.
  // (x-faces of the FP32 forms: from the slabs the step kernel staged, which
  // lie in this kernel's order; the state itself would be read a grid row apart)
  const S* xs = (d == 0 && xst) ? xst + spp : nullptr;
  const long long xv = (long long)NS * P * plane;   // stride of a variable in xst
  // ring slot of level n - k - l (>= 1: delays start after L + T_l steps);
  // k + l <= L + M < nlev, so one wrap of (n mod nlev) - k - l suffices
  auto level_at = [&](int l, int v) {
    int rs = nm - k - l;
    if (rs < 0) rs += g.nlev;
    return ring[((long long)rs * 5 + v) * qstride + spp];
  };
  // every load of this ghost point first, all in flight together: level n of
  // the source point (with its low words) and, under a delay, the T_l ring
  // levels n-k .. n-k-M (slots other than that of level n, written below)
  S src_hi[5], src_lo[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    src_hi[v] = xs ? xs[v * xv] : U[v * N + src];
    src_lo[v] = xs ? (xst_half ? xs[xst_half + v * xv] : S(0)) : (Ulo ? Ulo[v * N + src] : S(0));
  }
  double lv[M + 1][5];
  if (k > 0) {
#pragma unroll
    for (int l = 0; l <= M; ++l)
#pragma unroll
      for (int v = 0; v < 5; ++v) lv[l][v] = level_at(l, v);
  }
  {
    double* rw = ring + (long long)nm * 5 * qstride + spp;
#pragma unroll
    for (int v = 0; v < 5; ++v) rw[(long long)v * NS * P * plane] = ring_value(src_hi[v], src_lo[v]);
  }
  if (k == 0) {
    if (PQ) {
      // the derived fields of level n already exist (multi-pass path)
      out[0] = U[(1 + d) * N + src];
#pragma unroll
      for (int e = 1; e < 5; ++e) out[e * qstride] = PQ[(4 + 4 * d + e - 1) * N + src];
#pragma unroll
      for (int q = 0; q < 4; ++q) out[(5 + q) * qstride] = PQ[q * N + src];
    } else {
      S q[kNumGhostQ];
      ghost_quantities(K, d, src_hi, q);
#pragma unroll
      for (int qq = 0; qq < kNumGhostQ; ++qq) out[qq * qstride] = q[qq];
    }
    return;
  }
  int wi[M + 1];
  at_weights<M>(k, wi);
  if (g.xstate) {
    // the other reading of Table B's extrapolation: the state U extrapolated
    // to level n, sum_l w_l U^{n-k-l}, and the quantities evaluated once
    S Ux[5];
    if constexpr (sizeof(S) == 8) {
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        S a = S(wi[0]) * lv[0][v];
#pragma unroll
        for (int l = 1; l <= M; ++l) a = fma(S(wi[l]), lv[l][v], a);
        Ux[v] = a;
      }
    } else {
      // FP32: B + sum_l w_l (U_l - B) with B = level n-k truncated to FP32
      // (the weights sum to one), each difference formed as in the
      // quantity reading below, so that rounding stays relative to U and to
      // the differences
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        float hb, lo, hi, lo2;
        split_double(lv[0][v], hb, lo);
        float e = (float)wi[0] * lo;
#pragma unroll
        for (int l = 1; l <= M; ++l) {
          split_double(lv[l][v], hi, lo2);
          e = fmaf((float)wi[l], (hi - hb) + lo2, e);
        }
        Ux[v] = hb + e;
      }
    }
    S q[kNumGhostQ];
    ghost_quantities(K, d, Ux, q);
#pragma unroll
    for (int qq = 0; qq < kNumGhostQ; ++qq) out[qq * qstride] = q[qq];
    return;
  }
  S acc[kNumGhostQ];
  if constexpr (sizeof(S) == 8) {
#pragma unroll
    for (int q = 0; q < kNumGhostQ; ++q) acc[q] = S(0);
#pragma unroll
    for (int l = 0; l <= M; ++l) {
      const S w = S(wi[l]);
      S Uv[5], q[kNumGhostQ];
#pragma unroll
      for (int v = 0; v < 5; ++v) Uv[v] = lv[l][v];
      ghost_quantities(K, d, Uv, q);
#pragma unroll
      for (int qq = 0; qq < kNumGhostQ; ++qq) acc[qq] = fma(w, q[qq], acc[qq]);
    }
  } else {
    // base B = level n-k truncated to FP32; its own remainder is level 0's dU
    float h0, h1, h2, h3, h4, l0, l1, l2, l3, l4;
    split_double(lv[0][0], h0, l0);
    split_double(lv[0][1], h1, l1);
    split_double(lv[0][2], h2, l2);
    split_double(lv[0][3], h3, l3);
    split_double(lv[0][4], h4, l4);
    const GhostBase B = ghost_base(K, h0, h1, h2, h3, h4);
    {
      const float hb[5] = {h0, h1, h2, h3, h4};
      S q[kNumGhostQ];
      ghost_quantities(K, d, hb, q);
#pragma unroll
      for (int qq = 0; qq < kNumGhostQ; ++qq) acc[qq] = q[qq];
    }
    ghost_delta_f32(K, d, B, l0, l1, l2, l3, l4, (float)wi[0], acc);
#pragma unroll
    for (int l = 1; l <= M; ++l) {
      float hi, lo, dv[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        split_double(lv[l][v], hi, lo);
        const float hb = v == 0 ? h0 : (v == 1 ? h1 : (v == 2 ? h2 : (v == 3 ? h3 : h4)));
        dv[v] = (hi - hb) + lo;
      }
      ghost_delta_f32(K, d, B, dv[0], dv[1], dv[2], dv[3], dv[4], (float)wi[l], acc);
    }
  }
#pragma unroll
  for (int q = 0; q < kNumGhostQ; ++q) out[q * qstride] = acc[q];
}

template <typename S, int M>
__global__ void __launch_bounds__(256) k_ghost(Geom g, Coef<S> K, const S* __restrict__ U0,
                                               const S* __restrict__ U1, const S* __restrict__ Ulo0,
                                               const S* __restrict__ Ulo1, const DevState* __restrict__ ds,
                                               const S* __restrict__ PQ, S* GH0, S* GH1, S* GH2,
                                               double* __restrict__ ring0, double* __restrict__ ring1,
                                               double* __restrict__ ring2, const S* __restrict__ xst,
                                               long long xst_half, const uint8_t* __restrict__ dmap,
                                               long long n, long long cnt0, long long cnt1, long long cnt2) {
  const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  ghost_point<S, M>(g, K, U0, U1, Ulo0, Ulo1, ds, PQ, GH0, GH1, GH2, ring0, ring1, ring2, xst, xst_half,
                    [&](int p, int face) { return (int)dmap[p * 6 + face]; }, n, cnt0, cnt1, cnt2, j);
}

// ---------------------------------------------------------------------------
struct Pt {
  long long idx;
  int c[3], li[3], pe[3];
  long long pl[3];
};

__device__ __forceinline__ Pt make_point(const Geom& g, long long idx) {
  Pt P;
  P.idx = idx;
  decode(g, idx, P.c[0], P.c[1], P.c[2]);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    P.pe[d] = P.c[d] / g.nl[d];
    P.li[d] = P.c[d] - P.pe[d] * g.nl[d];
    P.pl[d] = plane_index(g, d, P.c[0], P.c[1], P.c[2]);
  }
  return P;
}

// Neighbours of one point along direction d at offsets -M .. -1, +1 .. +M
// (entry j is offset j - M for j < M, j - M + 1 above): either an offset into
// the field relative to the point (inside the PE, or periodic wrap when the
// direction has one PE) or, across a PE face, an index into the ghost array of
// direction d.  Built once per point and direction, then used for every
// quantity of that direction.  Offsets and indices are 32-bit: grids hold
// fewer than 2^31 points and a ghost array fewer than the grid.
template <int M>
struct Nb {
  int off[2 * M];
  unsigned gmask;    // bit j: off[j] indexes the ghost array
};

template <int M>
__device__ __forceinline__ Nb<M> make_nb(const Geom& g, const Pt& P, int d) {
  Nb<M> nb;
  nb.gmask = 0;
  const int st = (int)g.stride[d];
#pragma unroll
  for (int j = 0; j < 2 * M; ++j) {
    const int m = j < M ? j - M : j - M + 1;
    if (g.pes[d] == 1) {
      int c2 = P.c[d] + m;
      c2 = c2 < 0 ? c2 + g.n[d] : (c2 >= g.n[d] ? c2 - g.n[d] : c2);
      nb.off[j] = (c2 - P.c[d]) * st;
    } else {
      const int l2 = P.li[d] + m;
      if (l2 >= 0 && l2 < g.nl[d]) {
        nb.off[j] = m * st;
      } else {
        const int slot = l2 < 0 ? l2 + M : M + (l2 - g.nl[d]);
        nb.off[j] = (2 * M * P.pe[d] + slot) * (int)g.plane[d] + (int)P.pl[d];
        nb.gmask |= 1u << j;
      }
    }
  }
  return nb;
}

// Neighbour j of quantity f (ghost array gh across a face).  G = false: no
// lane of the warp has a ghost neighbour in this direction (a warp-uniform
// fact, tested with a vote), so the field is read directly.
template <bool G, typename S, int M>
__device__ __forceinline__ S nbv(const Nb<M>& nb, int j, int idx, const S* __restrict__ f,
                                 const S* __restrict__ gh) {
  if constexpr (!G) return f[idx + nb.off[j]];
  return ((nb.gmask >> j) & 1u) ? gh[nb.off[j]] : f[idx + nb.off[j]];
}

// acc - D1 f or acc + D1 f (sign s = -1 or 1 folded into the coefficients)
// with D1 = sum_m c_m (f[+m]-f[-m])  (differences first: rounding relative to
// the derivative, not to the stencil terms).  Entry M - 1 + m is offset +m,
// entry M - m is offset -m.
template <bool G, typename S, int M>
__device__ __forceinline__ S nb_d1_acc(S acc, S c1, S c2, S c3, const Nb<M>& nb, int idx, const S* f,
                                       const S* gh) {
  acc = fma(c1, nbv<G>(nb, M, idx, f, gh) - nbv<G>(nb, M - 1, idx, f, gh), acc);
  acc = fma(c2, nbv<G>(nb, M + 1, idx, f, gh) - nbv<G>(nb, M - 2, idx, f, gh), acc);
  if constexpr (M == 3) acc = fma(c3, nbv<G>(nb, M + 2, idx, f, gh) - nbv<G>(nb, M - 3, idx, f, gh), acc);
  return acc;
}

// D2 without the centre term: sum_m a_m (f[+m]+f[-m]).
template <bool G, typename S, int M>
__device__ __forceinline__ S nb_d2_off(S a1, S a2, S a3, const Nb<M>& nb, int idx, const S* f, const S* gh) {
  if constexpr (M == 2)
    return fma(a1, nbv<G>(nb, 2, idx, f, gh) + nbv<G>(nb, 1, idx, f, gh),
               a2 * (nbv<G>(nb, 3, idx, f, gh) + nbv<G>(nb, 0, idx, f, gh)));
  return fma(a1, nbv<G>(nb, 3, idx, f, gh) + nbv<G>(nb, 2, idx, f, gh),
             fma(a2, nbv<G>(nb, 4, idx, f, gh) + nbv<G>(nb, 1, idx, f, gh),
                 a3 * (nbv<G>(nb, 5, idx, f, gh) + nbv<G>(nb, 0, idx, f, gh))));
}

template <bool B>
struct BoolC {
  static constexpr bool value = B;
};

// Run body(BoolC<G>) with G = whether any active lane of the warp reads a
// ghost in this direction (warp-uniform branch: both loads of the select are
// issued only where a face is near).
template <int M, typename F>
__device__ __forceinline__ void with_ghosts(const Nb<M>& nb, F&& body) {
  if (__any_sync(__activemask(), nb.gmask != 0u)) body(BoolC<true>{});
  else body(BoolC<false>{});
}

template <typename S, int M>
__global__ void __launch_bounds__(256) k_grad(Geom g, Coef<S> K, const S* __restrict__ PQ,
                                              const S* __restrict__ GH0, const S* __restrict__ GH1,
                                              const S* __restrict__ GH2, S* __restrict__ G) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= g.npts) return;
  const Pt P = make_point(g, idx);
  const long long N = g.npts;
  const int i32 = (int)idx;
  const S* GH[3] = {GH0, GH1, GH2};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const long long qs = 2LL * M * g.pes[d] * g.plane[d];
    const Nb<M> nb = make_nb<M>(g, P, d);
    with_ghosts(nb, [&](auto gh_) {
      constexpr bool Gh = decltype(gh_)::value;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const S v = nb_d1_acc<Gh, S, M>(S(0), K.c1[d], K.c2[d], K.c3[d], nb, i32, PQ + q * N, GH[d] + (5 + q) * qs);
        const int out = q < 3 ? 3 * q + d : 9 + d;
        G[out * N + idx] = v;
      }
    });
  }
}

// ---------------------------------------------------------------------------
// Mixed-derivative helpers (Sec. 2.1).

// Kind of the PE-local first-derivative stencil at a point (kLocalOff /
// kLocal6Off rows): 0 central; 1 .. M the first M points of a PE; M+1 .. 2M
// the last M points.
template <int M>
__device__ __forceinline__ int local_kind_of(const Geom& g, const Pt& P, int d) {
  if (g.pes[d] == 1) return 0;
  const int li = P.li[d], nl = g.nl[d];
  if (li >= M && li <= nl - 1 - M) return 0;
  return li < M ? 1 + li : 1 + M + (li - (nl - M));
}

// PE-local first derivative of a gradient field in direction a: a
// table-driven loop, so only the one stencil that applies is evaluated.
template <typename S, int M>
__device__ __noinline__ S local_d1_table(const Geom& g, const Coef<S>& K, const Pt& P, int a, const S* __restrict__ f,
                                         int kind) {
  const long long s = g.stride[a];
  S acc = S(0);
  for (int i = 0; i < 2 * M + 1; ++i) {
    const S c = local_coefm<M>(S(0), kind, i);
    int off = local_off<M>(kind, i);
    if (g.pes[a] == 1) {   // central with periodic wrap
      int c2 = P.c[a] + off;
      c2 = c2 < 0 ? c2 + g.n[a] : (c2 >= g.n[a] ? c2 - g.n[a] : c2);
      off = c2 - P.c[a];
    }
    acc = fma(c, f[P.idx + (long long)off * s], acc);
  }
  return acc * K.hloc[a];
}

// PE-local 4th-order first derivative with the stencil written out per kind
// (the FP32 form: cheaper than the table when the FP64 pipe is not the limit).
template <typename S>
__device__ __forceinline__ S local_d1(const Geom& g, const Coef<S>& K, const Pt& P, int a, const S* __restrict__ f) {
  const long long s = g.stride[a];
  const long long i = P.idx;
  const int kind = local_kind_of<2>(g, P, a);
  if (kind == 0) {
    if (g.pes[a] == 1) {
      auto at = [&](int off) {
        int c2 = P.c[a] + off;
        c2 = c2 < 0 ? c2 + g.n[a] : (c2 >= g.n[a] ? c2 - g.n[a] : c2);
        return f[i + (long long)(c2 - P.c[a]) * s];
      };
      return fma(K.c1[a], at(1) - at(-1), K.c2[a] * (at(2) - at(-2)));
    }
    return fma(K.c1[a], f[i + s] - f[i - s], K.c2[a] * (f[i + 2 * s] - f[i - 2 * s]));
  }
  const S h = K.hloc[a];
  if (kind == 1)
    return h * (S(-25) * f[i] + S(48) * f[i + s] - S(36) * f[i + 2 * s] + S(16) * f[i + 3 * s] - S(3) * f[i + 4 * s]);
  if (kind == 2)
    return h * (S(-3) * f[i - s] - S(10) * f[i] + S(18) * f[i + s] - S(6) * f[i + 2 * s] + f[i + 3 * s]);
  if (kind == 3)
    return h * (S(3) * f[i + s] + S(10) * f[i] - S(18) * f[i - s] + S(6) * f[i - 2 * s] - f[i - 3 * s]);
  return h * (S(25) * f[i] - S(48) * f[i - s] + S(36) * f[i - 2 * s] - S(16) * f[i - 3 * s] + S(3) * f[i - 4 * s]);
}

// d/dx_a (d f/dx_b) with Gb = AT df/dx_b and Ga = AT df/dx_a (Sec. 2.1): the
// central derivative in a of Gb inside (fast path), the average of the two
// PE-local derivatives at PE-boundary points.  The FP64 form (and the 6th-order
// scheme) evaluates the one-sided stencils from a table out of line (fewer
// FP64-pipe instructions); the 4th-order FP32 form keeps them inline.
template <typename S, int M>
__device__ __forceinline__ S mixed(const Geom& g, const Coef<S>& K, const Pt& P, int a, int b, const S* Gb,
                                   const S* Ga) {
  if constexpr (sizeof(S) == 4 && M == 2) {
    if (local_kind_of<2>(g, P, a) == 0 && local_kind_of<2>(g, P, b) == 0) return local_d1(g, K, P, a, Gb);
    return S(0.5) * (local_d1(g, K, P, a, Gb) + local_d1(g, K, P, b, Ga));
  }
  const int ka = local_kind_of<M>(g, P, a), kb = local_kind_of<M>(g, P, b);
  if (ka == 0 && kb == 0 && g.pes[a] > 1) {
    const long long s = g.stride[a], i = P.idx;
    if constexpr (M == 2) return fma(K.c1[a], Gb[i + s] - Gb[i - s], K.c2[a] * (Gb[i + 2 * s] - Gb[i - 2 * s]));
    return fma(K.c1[a], Gb[i + s] - Gb[i - s],
               fma(K.c2[a], Gb[i + 2 * s] - Gb[i - 2 * s], K.c3[a] * (Gb[i + 3 * s] - Gb[i - 3 * s])));
  }
  if (ka == 0 && kb == 0) return local_d1_table<S, M>(g, K, P, a, Gb, 0);
  return S(0.5) * (local_d1_table<S, M>(g, K, P, a, Gb, ka) + local_d1_table<S, M>(g, K, P, b, Ga, kb));
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_min(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Order-preserving integer keys (min/max without floating-point compares).
__device__ __forceinline__ long long okey(double v) { return ordered_key(v); }
__device__ __forceinline__ long long okey(float v) {
  // the float key is widened to the double key of the same value on the
  // host side only after decoding, so encode through the exact double value
  const int b = __float_as_int(v);
  return (long long)(b ^ ((b >> 31) & 0x7FFFFFFF));
}

// (hi, lo) += (bh, bl) in double-float arithmetic: TwoSum of the high words
// (Knuth), low words and the rounding error summed, then renormalised.
__device__ __forceinline__ void df_add(float& hi, float& lo, float bh, float bl) {
  const float s = __fadd_rn(hi, bh);
  const float bp = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(bh, bp));
  const float l = __fadd_rn(__fadd_rn(lo, bl), e);
  hi = __fadd_rn(s, l);
  lo = __fsub_rn(l, __fsub_rn(hi, s));
}

// Per-block reduction of the kNumStat per-thread sums (fixed order) into
// partial[block], and of the max/min keys and health bits into the global
// words.  Blocks have a multiple of 32 threads, at most NT.  Each statistic
// goes through shared memory in NT/16 partial sums of 16 threads, then one sum
// of those (a warp-shuffle tree would cost every lane 5 adds per statistic).
// FP64 values are summed in FP64.  FP32 values arrive as (sum, compensation)
// pairs and are summed as double-float pairs (about 48 significant bits) in
// FP32 arithmetic, so that only the last sum of each statistic touches the
// FP64 pipe.
constexpr int kReduceScratchDoubles = kNumStat * 257;   // NT = 256

// scratch: at least kNumStat * (NT + 1) doubles of shared memory that no
// other thread of the block still reads (k_fused passes its dead window).
// stc: the compensations of the FP32 sums (sum - stc is the compensated sum;
// null: none).
template <typename S, int NT = 256>
__device__ __forceinline__ void block_reduce(S (&st)[kNumStat], long long kwave, long long krho, long long kp,
                                             unsigned health, bool do_stats, double* partial,
                                             unsigned long long* words, double* scratch,
                                             const S* stc = nullptr, long long blk_index = -1) {
  constexpr int kMaxThreads = NT, kMaxWarps = kMaxThreads / 32, kParts = kMaxThreads / 16;
  double (*sh)[kMaxThreads + 1] = reinterpret_cast<double (*)[kMaxThreads + 1]>(scratch);
  float2 (*shp)[kMaxThreads + 1] = reinterpret_cast<float2 (*)[kMaxThreads + 1]>(scratch);   // FP32 pairs
  __shared__ long long shk[kMaxWarps][3];
  __shared__ unsigned shh[kMaxWarps];
  const int nthreads = blockDim.x * blockDim.y * blockDim.z;
  const int nwarps = nthreads >> 5;
  const int tid = (threadIdx.z * blockDim.y + threadIdx.y) * blockDim.x + threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5;
  const long long blk =
      blk_index >= 0 ? blk_index : ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  const unsigned hh = __reduce_or_sync(0xffffffffu, health);
  const bool by_warp = sizeof(S) == 4;
  if (do_stats) {
    kwave = warp_max(kwave);
    krho = warp_min(krho);
    kp = warp_min(kp);
    if (lane == 0) { shk[wid][0] = kwave; shk[wid][1] = krho; shk[wid][2] = kp; }
    if (!by_warp) {
#pragma unroll
      for (int s = 0; s < kNumStat; ++s) sh[s][tid] = (double)st[s];
      for (int j = nthreads + tid; j < kMaxThreads; j += nthreads)
#pragma unroll
        for (int s = 0; s < kNumStat; ++s) sh[s][j] = 0.0;
    } else {
      // stays FP32 here: a conversion to FP64 is an FP64-pipe warp
      // instruction even with one active lane
#pragma unroll
      for (int s = 0; s < kNumStat; ++s) shp[s][tid] = make_float2((float)st[s], stc ? -(float)stc[s] : 0.f);
      for (int j = nthreads + tid; j < kMaxThreads; j += nthreads)
#pragma unroll
        for (int s = 0; s < kNumStat; ++s) shp[s][j] = make_float2(0.f, 0.f);
    }
  }
  if (lane == 0) shh[wid] = hh;
  __syncthreads();
  if (tid == 0) {
    unsigned h = 0;
    for (int w = 0; w < nwarps; ++w) h |= shh[w];
    if (h) atomicOr((unsigned*)(words + 3), h);
    if (do_stats) {
      long long kw = LLONG_MIN, kr = LLONG_MAX, kq = LLONG_MAX;
      for (int w = 0; w < nwarps; ++w) {
        kw = max(kw, shk[w][0]); kr = min(kr, shk[w][1]); kq = min(kq, shk[w][2]);
      }
      atomicMax((long long*)(words + 0), kw);
      atomicMin((long long*)(words + 1), kr);
      atomicMin((long long*)(words + 2), kq);
    }
  }
  if (!do_stats) return;
  if (!by_warp) {
    // 16 consecutive entries per (statistic, part), written back in place
    for (int j = tid; j < kNumStat * kParts; j += nthreads) {
      const int s = j / kParts, part = j - s * kParts;
      double a = 0.0;
#pragma unroll
      for (int q = 0; q < 16; ++q) a += sh[s][part * 16 + q];
      sh[s][part * 16] = a;
    }
    __syncthreads();
    for (int s = tid; s < kNumStat; s += nthreads) {
      double a = 0.0;
#pragma unroll
      for (int part = 0; part < kParts; ++part) a += sh[s][part * 16];
      partial[blk * kNumStat + s] = a;
    }
  } else {
    for (int j = tid; j < kNumStat * kParts; j += nthreads) {
      const int s = j / kParts, part = j - s * kParts;
      float2 a = shp[s][part * 16];
#pragma unroll
      for (int q = 1; q < 16; ++q) {
        const float2 b = shp[s][part * 16 + q];
        df_add(a.x, a.y, b.x, b.y);
      }
      shp[s][part * 16] = a;
    }
    __syncthreads();
    // one warp: the parts as a pair, then hi + lo once in FP64
    for (int s = tid; s < kNumStat; s += nthreads) {
      float2 a = shp[s][0];
      for (int part = 1; part < kParts; ++part) {
        const float2 b = shp[s][part * 16];
        df_add(a.x, a.y, b.x, b.y);
      }
      partial[blk * kNumStat + s] = (double)a.x + (double)a.y;
    }
  }
}

// ---------------------------------------------------------------------------
// Linear index of the point of this thread of k_main (blocks of 256).  When
// the block's 256 consecutive points are whole PE rows in x (PE width 8, 16
// or 32 divides 256 and the row length, so a full block starts at a row
// start), the points next to the two x-faces of every PE row go to the
// block's first warps and the interior points to the others, so that the
// one-sided stencils of the mixed rule run in those warps only instead of
// diverging in every warp (in the FP64 form a divergent path costs the whole
// warp on the FP64 pipe).
template <typename S>
__device__ __forceinline__ long long main_point_index(const Geom& g) {
  const long long base = blockIdx.x * (long long)blockDim.x;
  int t = threadIdx.x;
  {
    const int nl = g.nl[0];
    if (g.pes[0] > 1 && (nl == 8 || nl == 16 || nl == 32) && base + 256 <= g.npts) {
      const int nb = 4 * (256 / nl);   // face-adjacent points of the block: whole warps
      if (t < nb) {
        const int r = t >> 2, c = t & 3;
        t = r * nl + (c < 2 ? c : nl - 4 + c);
      } else {
        const int u = t - nb, w = nl - 4;
        const int r = u / w;
        t = r * nl + 2 + (u - r * w);
      }
    }
  }
  return base + t;
}

// FP64: three CTAs per SM (more warps to hide the FP64 pipe's latency; a
// few registers spill); FP32: two.
template <typename S, int M>
__global__ void __launch_bounds__(256, sizeof(S) == 8 ? 3 : 2) k_main(Geom g, Coef<S> K, StepArgs<S> A0) {
  const StepArgs<S>& A = A0;
  const StepDyn<S> D = resolve_step(A0);
  const long long idx = main_point_index<S>(g);
  const bool active = idx < g.npts;
  S st[kNumStat];
#pragma unroll
  for (int s = 0; s < kNumStat; ++s) st[s] = S(0);
  long long kwave = LLONG_MIN, krho = LLONG_MAX, kp = LLONG_MAX;
  unsigned health = 0;

  if (active) {
    const Pt P = make_point(g, idx);
    const long long N = g.npts;
    const S* U = D.U;
    const S* PQ = A.PQ;
    const S* G = A.G;

    // inviscid flux divergence -sum_d D_d F_d (accumulated with the stencil
    // coefficients negated) and the off-centre parts of the second
    // derivatives of u, v, w, T, direction by direction (AT ghosts across faces)
    S R[5] = {S(0), S(0), S(0), S(0), S(0)};
    S lap[4] = {S(0), S(0), S(0), S(0)};
    S d2diag[3];                           // d^2 u_d / dx_d^2
    S a0sum = S(0);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const long long qs = 2LL * M * g.pes[d] * g.plane[d];
      const Nb<M> nb = make_nb<M>(g, P, d);
      const S* gh = A.GH[d];
      const int i32 = (int)idx;
      with_ghosts(nb, [&](auto gh_) {
        constexpr bool Gh = decltype(gh_)::value;
#pragma unroll
        for (int e = 0; e < 5; ++e) {
          const S* f = e == 0 ? U + (1 + d) * N : PQ + (4 + 4 * d + e - 1) * N;
          R[e] = nb_d1_acc<Gh, S, M>(R[e], -K.c1[d], -K.c2[d], -K.c3[d], nb, i32, f, gh + e * qs);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const S v = nb_d2_off<Gh, S, M>(K.a1[d], K.a2[d], K.a3[d], nb, i32, PQ + q * N, gh + (5 + q) * qs);
          lap[q] += v;
          if (q == d) d2diag[d] = fma(K.a0[d], PQ[q * N + idx], v);
        }
      });
      a0sum += K.a0[d];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) lap[q] = fma(a0sum, PQ[q * N + idx], lap[q]);

    // first derivatives at the point
    S Ag[3][3], dT[3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) Ag[i][j] = G[(3 * i + j) * N + idx];
#pragma unroll
    for (int j = 0; j < 3; ++j) dT[j] = G[(9 + j) * N + idx];

    // d theta / dx_i = d2 u_i/dx_i^2 + sum_{k != i} d/dx_i (d u_k / dx_k)
    S gth[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      S s = d2diag[i];
#pragma unroll
      for (int k = 0; k < 3; ++k)
        if (k != i) s += mixed<S, M>(g, K, P, i, k, G + (3 * k + k) * N, G + (3 * k + i) * N);
      gth[i] = s;
    }

    const S r = U[idx];
    const S m[3] = {U[N + idx], U[2 * N + idx], U[3 * N + idx]};
    const S E = U[4 * N + idx];
    const S vel[3] = {PQ[idx], PQ[N + idx], PQ[2 * N + idx]};
    const S T = PQ[3 * N + idx];
    const S p = pressure(K, m[0], m[1], m[2], vel[0], vel[1], vel[2], E);
    const S theta = Ag[0][0] + Ag[1][1] + Ag[2][2];
    S mu, dmudT;
    viscosity(K, T, mu, dmudT);
    const S kappa = mu * K.cp_over_pr;
    S dmu[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) dmu[j] = dmudT * dT[j];

    S sm[3][3];   // A_ij + A_ji - 2/3 delta_ij theta
    const S th23 = S(2.0 / 3.0) * theta;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) sm[i][j] = i == j ? S(2) * Ag[i][i] - th23 : Ag[i][j] + Ag[j][i];

    // forcing f_c = sum_kx Re(B[kx][c](y,z) exp(i kx x))
    S fo[3] = {S(0), S(0), S(0)};
    if (A.fB) {
      const int x = P.c[0], y = P.c[1], z = P.c[2];
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

    // sigma_ij S_ij = mu/2 sum_ij sm_ij (A_ij + A_ji): diagonal terms
    // sm_ii A_ii, off-diagonal pairs sm_ij^2 (each counted twice, halved)
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
    // conduction k lap T + grad k . grad T, then the form's energy sources:
    // total E: viscous work u_i V_i + sigma S + forcing power; rho e (Eq. (ie)):
    // -p theta + sigma S
    const S heat = fma(K.cp_over_pr, fma(dmu[0], dT[0], fma(dmu[1], dT[1], dmu[2] * dT[2])), kappa * lap[3]);
    if (K.eform) R[4] += fma(-p, theta, sigS + heat);
    else R[4] += fma(r, fma(fo[0], vel[0], fma(fo[1], vel[1], fo[2] * vel[2])), sigS + work + heat);

    // health: rho <= 0, p <= 0, non-finite R (bit tests)
    if (nonpositive(r)) health |= H_RHO;
    if (nonpositive(p)) health |= H_P;
#pragma unroll
    for (int v = 0; v < 5; ++v)
      if (nonfinite(R[v])) health |= H_NONFINITE;

    if (A.do_update) {
      const S Uo[5] = {r, m[0], m[1], m[2], E};
      S un[5], unlo[5];
      ab2_update(K, A, D, idx, N, Uo, R, un, unlo, health);
      // (the ring slabs of level n+1 are written by the next step's ghost kernel)
      stage_xface(g, A, P.li[0], P.pe[0], P.pl[0], un, unlo);
    } else if (A.Rout) {
#pragma unroll
      for (int v = 0; v < 5; ++v) A.Rout[v * N + idx] = (double)R[v];
    }

    if (A.do_stats) {
      const S uu = fma(vel[0], vel[0], fma(vel[1], vel[1], vel[2] * vel[2]));
      const S c = sqrt(T);
      st[ST_RHO] = r;
      st[ST_M0] = m[0];
      st[ST_M1] = m[1];
      st[ST_M2] = m[2];
      st[ST_E] = E;
      st[ST_KE] = S(0.5) * r * uu;
      st[ST_SIGS] = sigS;
      const S a0 = Ag[0][0], a1 = Ag[1][1], a2 = Ag[2][2];
      const S q0 = a0 * a0, q1 = a1 * a1, q2 = a2 * a2;
      st[ST_G2] = q0 + q1 + q2;
      st[ST_G3] = fma(q0, a0, fma(q1, a1, q2 * a2));
      st[ST_G4] = fma(q0, q0, fma(q1, q1, q2 * q2));
      const S o0 = Ag[2][1] - Ag[1][2], o1 = Ag[0][2] - Ag[2][0], o2 = Ag[1][0] - Ag[0][1];
      st[ST_ENST] = fma(o0, o0, fma(o1, o1, o2 * o2));
      st[ST_PTHETA] = p * theta;
      st[ST_FPOW] = r * fma(fo[0], vel[0], fma(fo[1], vel[1], fo[2] * vel[2]));
      st[ST_U2] = uu;
      st[ST_C] = c;
      // max |u_d| + c: the largest |u_d| chosen by bit pattern (non-negative
      // values order as integers)
      const S au[3] = {abs_bits(vel[0]), abs_bits(vel[1]), abs_bits(vel[2])};
      const long long k0 = okey(au[0]), k1 = okey(au[1]), k2 = okey(au[2]);
      const S umax = (k0 >= k1 && k0 >= k2) ? au[0] : (k1 >= k2 ? au[1] : au[2]);
      kwave = okey(umax + c);
      krho = okey(r);
      kp = okey(p);
    }
  }
  __shared__ double red_scratch[kReduceScratchDoubles];
  block_reduce<S>(st, kwave, krho, kp, health, A.do_stats != 0, A.partial, A.words, red_scratch);
}

}  // namespace atdns
