// Device arithmetic of the PSDF (Sec. IV-A.3 stages 1-4), float32.
//
// Every operation that feeds a per-obstacle value is written with explicit
// round-to-nearest intrinsics (__fadd_rn, __fmul_rn, __fmaf_rn, ...), which
// the compiler may not contract or reassociate, so a value is the same bits
// wherever it is computed.
//
// Two candidate sets.  The scan (values only) takes the minimum over every
// clamped point-to-segment candidate, including the clamps that land on a
// segment's far end (a robot vertex to the next polygon vertex, an obstacle
// vertex to a robot vertex).  Each of those is a second copy of a candidate
// the set already holds exactly (Sec. IV-B: the endpoints are vertices, and
// a vertex-to-vertex distance is never below the vertex-to-edge distance of
// the edge that starts there), so the minimum changes by rounding at most,
// and the scan saves a compare and a select per robot vertex and edge.  The
// epilogue, which names the active pair, uses the exact candidate set: far-
// end clamps excluded, obstacle-vertex candidates only for interior
// projections.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "psdf_internal.h"

namespace psdf {

struct V2 {
  float x, y;
};

constexpr float kInf = __builtin_huge_valf();

// Stage 1: world -> robot-local frame, R(theta)^T (X - p).
__device__ __forceinline__ V2 to_local(float X, float Y, float px, float py, float c, float s)
{
  const float dx = __fsub_rn(X, px), dy = __fsub_rn(Y, py);
  V2 r;
  r.x = __fmaf_rn(c, dx, __fmul_rn(s, dy));
  r.y = __fmaf_rn(c, dy, -__fmul_rn(s, dx));
  return r;
}

// Edge vector B - A in the robot frame, rotated from the world-frame
// difference (exact or nearly so in FP32 for the endpoints of one edge)
// instead of taken between the two rotated endpoints: their rounding, about
// an ulp of their distance from the pose, would otherwise dominate the
// direction of a short edge (and the obstacle-axis overlaps built on it).
__device__ __forceinline__ V2 local_edge(float ax, float ay, float bx, float by, float c, float s)
{
  const float dx = __fsub_rn(bx, ax), dy = __fsub_rn(by, ay);
  V2 r;
  r.x = __fmaf_rn(c, dx, __fmul_rn(s, dy));
  r.y = __fmaf_rn(c, dy, -__fmul_rn(s, dx));
  return r;
}

// Programmatic dependent launch: a kernel launched with the programmatic
// stream-serialization attribute may start while its predecessor finishes;
// pdl_wait() blocks until the predecessor grid has completed and its memory is
// visible (a no-op for a kernel launched without the attribute), and
// pdl_trigger() lets the successor's launch begin once every CTA of this grid
// has passed it.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger()
{
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Requests every 128-byte line of [p, p + bytes) into L1 (at most 16 lines),
// so that the loads that follow, issued one after another by a dependent
// chain, hit L1 after a single memory latency.
__device__ __forceinline__ void prefetch_lines(const void *p, int bytes)
{
  const uintptr_t a0 = (uintptr_t)p & ~(uintptr_t)127, a1 = (uintptr_t)p + (uintptr_t)bytes;
  int n = 0;
  for (uintptr_t a = a0; a < a1 && n < 16; a += 128, ++n)
    asm volatile("prefetch.global.L1 [%0];" ::"l"(a));
}

// The same into L2 only.
__device__ __forceinline__ void prefetch_lines_l2(const void *p, int bytes)
{
  const uintptr_t a0 = (uintptr_t)p & ~(uintptr_t)127, a1 = (uintptr_t)p + (uintptr_t)bytes;
  int n = 0;
  for (uintptr_t a = a0; a < a1 && n < 16; a += 128, ++n)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
}

// Total order on float values as unsigned bits (-0 is folded onto +0 first
// so that the order matches IEEE comparison).
__device__ __forceinline__ uint32_t ordered_bits(float v)
{
  const uint32_t b = __float_as_uint(__fadd_rn(v, 0.0f));
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ float from_ordered_bits(uint32_t o)
{
  return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

// Min-key of one obstacle: (ordered value << 32) | rank, rank = the caller's
// row of the obstacle's first edge.  Its minimum over obstacles realises
// Eq. psdf_value with the lowest-rank tie-break.
__device__ __forceinline__ unsigned long long pack_key(float v, int rank)
{
  return ((unsigned long long)ordered_bits(v) << 32) | (unsigned)rank;
}

__device__ __forceinline__ unsigned make_pid(int edge, int kind, int l)
{
  return ((unsigned)edge << kPairShiftEdge) | ((unsigned)kind << kPairShiftKind) | (unsigned)l;
}

// Stage 4 (Sec. IV-D), hard penetration: value compared across obstacles.
// Separated -> squared distance (monotone in d); otherwise -max(delta_min, 0).
__device__ __forceinline__ float synth_value(float d2min, float dmin_axes, float eps_sat)
{
  const bool separated = dmin_axes < -eps_sat;
  return separated ? d2min : -fmaxf(dmin_axes, 0.0f);
}

// Soft minimum of Eq. penetration_depth over an obstacle's axes,
// pen = -(1/eta) log sum_n exp(-eta delta_+(n)), accumulated one axis at a
// time around the running minimum mu of delta_+ (every term <= 1):
// S = sum exp(-eta (delta_+ - mu)), pen = mu - log(S) / eta.  Explicit
// rounding, so the scan and the epilogue reach the same bits when they add
// the axes in the same order.
struct SoftAcc {
  float mu = kInf, S = 0.f;
  __device__ __forceinline__ void add(float delta, float eta)
  {
    const float x = fmaxf(delta, 0.f);
    if (x < mu) {
      S = __fmaf_rn(S, expf(__fmul_rn(-eta, __fsub_rn(mu, x))), 1.f);
      mu = x;
    } else {
      S = __fadd_rn(S, expf(__fmul_rn(-eta, __fsub_rn(x, mu))));
    }
  }
  __device__ __forceinline__ float pen(float eta) const
  {
    return __fsub_rn(mu, __fdiv_rn(logf(S), eta));
  }
};

// A non-separated soft value sd = -pen can be positive (shallow overlaps,
// Sec. IV-D); mapped like the squared separation so that one ordering holds
// across separated (d^2) and non-separated obstacles.
__device__ __forceinline__ float soft_key(float sd)
{
  return sd > 0.f ? __fmul_rn(sd, sd) : sd;
}

// ---------------------------------------------------------------------------
// footprint access
// ---------------------------------------------------------------------------
// The constants one edge step reads for robot vertex l.
struct RobotL {
  float vx, vy, ex, ey, inv_e2, nx, ny;
};

// A footprint passed by value as a kernel parameter: the loads below become
// constant-bank operands of the arithmetic.
__device__ __forceinline__ RobotL robot_l(const FootprintK &F, int l)
{
  return RobotL{F.vx[l], F.vy[l], F.ex[l], F.ey[l], F.inv_e2[l], F.nx[l], F.ny[l]};
}

__device__ __forceinline__ float2 robot_interval(const FootprintK &F, int l)
{
  return make_float2(F.alo[l], F.ahi[l]);
}

// The constants of robot vertices 2q and 2q + 1 as pairs, for the paired
// FP32 instructions of the edge step (inv_e2 negated).
struct RobotL2 {
  float2 vx, vy, ex, ey, nie, nx, ny;
};

__device__ __forceinline__ RobotL2 robot_l2(const FootprintK &F, int q)
{
  const int a = 2 * q, b = 2 * q + 1;
  return RobotL2{make_float2(F.vx[a], F.vx[b]),          make_float2(F.vy[a], F.vy[b]),
                 make_float2(F.ex[a], F.ex[b]),          make_float2(F.ey[a], F.ey[b]),
                 make_float2(-F.inv_e2[a], -F.inv_e2[b]), make_float2(F.nx[a], F.nx[b]),
                 make_float2(F.ny[a], F.ny[b])};
}

// A footprint staged in shared memory as records (one per robot vertex:
// {vx, vy, ex, ey}, {inv_e2, nx, ny, 0}; intervals {alo, ahi}), for kernels
// whose CTAs change footprint from one work item to the next.  The loads are
// volatile, so they are re-issued at every use (two 16-byte broadcasts per
// robot vertex and edge) instead of the compiler holding all constants of a
// large footprint in registers across the obstacle loop.
struct FootprintS {
  const float4 *rec;   // [2 * m]
  const float2 *ivl;   // [m]
  const float4 *pair;  // [4 * (m / 2)]: {vx, vx', vy, vy'}, {ex, ex', ey, ey'},
                       // {-inv_e2, -inv_e2', nx, nx'}, {ny, ny', 0, 0}
};

__device__ __forceinline__ float4 lds_f4(const float4 *p)
{
  float4 r;
  asm volatile("ld.volatile.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
               : "r"((unsigned)__cvta_generic_to_shared(p)));
  return r;
}

__device__ __forceinline__ float2 lds_f2(const float2 *p)
{
  float2 r;
  asm volatile("ld.volatile.shared.v2.f32 {%0, %1}, [%2];"
               : "=f"(r.x), "=f"(r.y)
               : "r"((unsigned)__cvta_generic_to_shared(p)));
  return r;
}

__device__ __forceinline__ RobotL robot_l(const FootprintS &F, int l)
{
  const float4 a = lds_f4(F.rec + 2 * l), b = lds_f4(F.rec + 2 * l + 1);
  return RobotL{a.x, a.y, a.z, a.w, b.x, b.y, b.z};
}

__device__ __forceinline__ float2 robot_interval(const FootprintS &F, int l)
{
  return lds_f2(F.ivl + l);
}

__device__ __forceinline__ RobotL2 robot_l2(const FootprintS &F, int q)
{
  const float4 a = lds_f4(F.pair + 4 * q), b = lds_f4(F.pair + 4 * q + 1);
  const float4 c = lds_f4(F.pair + 4 * q + 2), d = lds_f4(F.pair + 4 * q + 3);
  return RobotL2{make_float2(a.x, a.y), make_float2(a.z, a.w), make_float2(b.x, b.y),
                 make_float2(b.z, b.w), make_float2(c.x, c.y), make_float2(c.z, c.w),
                 make_float2(d.x, d.y)};
}

// ---------------------------------------------------------------------------
// value-only evaluation of one obstacle (the scan's inner loop)
// ---------------------------------------------------------------------------
// One robot vertex against the edge A -> B (local frame): the distance from
// the vertex to the edge (Sec. IV-B d_v), from the edge's start vertex A to
// the robot edge (d_e), the vertex's offset on the edge axis (smin/smax)
// and A's projection on the robot axis (pmax/pmin).
template <bool SEG>
__device__ __forceinline__ void vertex_step(const RobotL &r, V2 A, V2 B, float ux, float uy,
                                            float inv_len2, float &smin, float &smax,
                                            float &d2min, float &pmax_l, float &pmin_l)
{
  // robot vertex l -> obstacle edge: t = clamp((v - A).u / (|u|^2 + eps))
  const float wx = __fsub_rn(r.vx, A.x), wy = __fsub_rn(r.vy, A.y);
  const float t = __saturatef(__fmul_rn(__fmaf_rn(wx, ux, __fmul_rn(wy, uy)), inv_len2));
  float rx = __fmaf_rn(-t, ux, wx), ry = __fmaf_rn(-t, uy, wy);
  if (SEG) {
    // a segment's far endpoint is its own vertex: use it exactly
    rx = (t == 1.0f) ? __fsub_rn(r.vx, B.x) : rx;
    ry = (t == 1.0f) ? __fsub_rn(r.vy, B.y) : ry;
  }
  const float d2 = __fmaf_rn(rx, rx, __fmul_rn(ry, ry));
  // robot vertex projected on rot90(u), measured from A (obstacle axis)
  const float sl = __fmaf_rn(wy, ux, -__fmul_rn(wx, uy));
  smin = fminf(smin, sl);
  smax = fmaxf(smax, sl);
  // obstacle vertex A -> robot edge l, t' = clamp((A - v).e / (|e|^2 + eps))
  const float tp = __saturatef(__fmul_rn(-__fmaf_rn(wx, r.ex, __fmul_rn(wy, r.ey)), r.inv_e2));
  const float qx = __fmaf_rn(tp, r.ex, wx), qy = __fmaf_rn(tp, r.ey, wy);
  const float d2p = __fmaf_rn(qx, qx, __fmul_rn(qy, qy));
  d2min = fminf(d2min, fminf(d2, d2p));
  // obstacle vertex A on the robot axis n_l
  const float pr = __fmaf_rn(A.x, r.nx, __fmul_rn(A.y, r.ny));
  pmax_l = fmaxf(pmax_l, pr);
  pmin_l = fminf(pmin_l, pr);
}

// One edge of a closed polygon, from A (= vertex k, local) to B (= vertex
// k+1, local).  Accumulates: d2min (squared separation, Sec. IV-B), the
// obstacle's projections on the robot axes (pmax/pmin, Sec. IV-C) and
// returns the overlap on this edge's own axis.  Robot vertices are taken in
// pairs on Blackwell's paired FP32 instructions (fma/add/mul .f32x2: two
// operations per issue slot; the clamps and minima stay scalar).  Every
// paired operation is the single-vertex operation with the same operands
// (a - b as a + (-b), -x * y as x * (-y)), so the results carry the same bits
// as vertex_step.
template <int M, bool SEG, class FP>
__device__ __forceinline__ float edge_step(const FP &F, V2 A, V2 B, V2 U, float inv_len2,
                                           float inv_len, float alpha_p, float beta_p,
                                           float (&pmax)[M], float (&pmin)[M], float &d2min)
{
  const float ux = U.x, uy = U.y;
  float smin = kInf, smax = -kInf;
  const float2 nax = make_float2(-A.x, -A.x), nay = make_float2(-A.y, -A.y);
  const float2 ax2 = make_float2(A.x, A.x), ay2 = make_float2(A.y, A.y);
  const float2 ux2 = make_float2(ux, ux), uy2 = make_float2(uy, uy);
  const float2 nux2 = make_float2(-ux, -ux), nuy2 = make_float2(-uy, -uy);
  const float2 il2 = make_float2(inv_len2, inv_len2);
#pragma unroll
  for (int q = 0; q < M / 2; ++q) {
    const RobotL2 r = robot_l2(F, q);
    const float2 wx = __fadd2_rn(r.vx, nax), wy = __fadd2_rn(r.vy, nay);
    const float2 tt = __fmul2_rn(__ffma2_rn(wx, ux2, __fmul2_rn(wy, uy2)), il2);
    const float2 t = make_float2(__saturatef(tt.x), __saturatef(tt.y));
    float2 rx = __ffma2_rn(t, nux2, wx), ry = __ffma2_rn(t, nuy2, wy);
    if (SEG) {
      const float2 bx = __fadd2_rn(r.vx, make_float2(-B.x, -B.x));
      const float2 by = __fadd2_rn(r.vy, make_float2(-B.y, -B.y));
      rx.x = (t.x == 1.0f) ? bx.x : rx.x;
      rx.y = (t.y == 1.0f) ? bx.y : rx.y;
      ry.x = (t.x == 1.0f) ? by.x : ry.x;
      ry.y = (t.y == 1.0f) ? by.y : ry.y;
    }
    const float2 d2 = __ffma2_rn(rx, rx, __fmul2_rn(ry, ry));
    const float2 sl = __ffma2_rn(wy, ux2, __fmul2_rn(wx, nuy2));
    smin = fminf(smin, fminf(sl.x, sl.y));
    smax = fmaxf(smax, fmaxf(sl.x, sl.y));
    const float2 tq = __fmul2_rn(__ffma2_rn(wx, r.ex, __fmul2_rn(wy, r.ey)), r.nie);
    const float2 tp = make_float2(__saturatef(tq.x), __saturatef(tq.y));
    const float2 qx = __ffma2_rn(tp, r.ex, wx), qy = __ffma2_rn(tp, r.ey, wy);
    const float2 d2p = __ffma2_rn(qx, qx, __fmul2_rn(qy, qy));
    d2min = fminf(d2min, fminf(fminf(d2.x, d2p.x), fminf(d2.y, d2p.y)));
    const float2 pr = __ffma2_rn(ax2, r.nx, __fmul2_rn(ay2, r.ny));
    pmax[2 * q] = fmaxf(pmax[2 * q], pr.x);
    pmax[2 * q + 1] = fmaxf(pmax[2 * q + 1], pr.y);
    pmin[2 * q] = fminf(pmin[2 * q], pr.x);
    pmin[2 * q + 1] = fminf(pmin[2 * q + 1], pr.y);
  }
  if (M & 1)
    vertex_step<SEG>(robot_l(F, M - 1), A, B, ux, uy, inv_len2, smin, smax, d2min, pmax[M - 1],
                     pmin[M - 1]);
  // overlap on this edge's axis: obstacle interval [alpha', beta'] vs the
  // robot interval [smin, smax] / (|u| + eps)
  const float da = __fmaf_rn(-smin, inv_len, beta_p);
  const float db = __fmaf_rn(smax, inv_len, -alpha_p);
  return fminf(da, db);
}

// A segment's B endpoint as an extra obstacle vertex: robot-edge distances
// and robot-axis projections.
template <int M, class FP>
__device__ __forceinline__ void extra_vertex(const FP &F, V2 X, float (&pmax)[M],
                                             float (&pmin)[M], float &d2min)
{
#pragma unroll
  for (int l = 0; l < M; ++l) {
    const RobotL r = robot_l(F, l);
    const float wx = __fsub_rn(r.vx, X.x), wy = __fsub_rn(r.vy, X.y);
    const float tp = __saturatef(__fmul_rn(-__fmaf_rn(wx, r.ex, __fmul_rn(wy, r.ey)), r.inv_e2));
    const float qx = __fmaf_rn(tp, r.ex, wx), qy = __fmaf_rn(tp, r.ey, wy);
    const float d2p = __fmaf_rn(qx, qx, __fmul_rn(qy, qy));
    d2min = fminf(d2min, d2p);
    const float pr = __fmaf_rn(X.x, r.nx, __fmul_rn(X.y, r.ny));
    pmax[l] = fmaxf(pmax[l], pr);
    pmin[l] = fminf(pmin[l], pr);
  }
}

// Value of one obstacle whose vertex records start at vt (2 float4 per vertex),
// in the min-key domain: d^2 when separated, else -pen (hard: the minimum
// of max(delta, 0); SOFT: Eq. penetration_depth with sharpness eta, through
// soft_key).  Axes are visited in a fixed order: each edge's own axis, then
// the robot axes.
template <int M, class FP, bool SOFT = false>
__device__ __forceinline__ float obstacle_value(const FP &F, float px, float py,
                                                float c, float s, const float4 *vt, int n,
                                                float eps_sat, float eta = 0.f)
{
  float pmax[M], pmin[M];
#pragma unroll
  for (int l = 0; l < M; ++l) {
    pmax[l] = -kInf;
    pmin[l] = kInf;
  }
  float d2min = kInf, dlt = kInf;
  SoftAcc acc;
  const float4 a0 = vt[0], b0 = vt[1];
  const V2 A0 = to_local(a0.x, a0.y, px, py, c, s);
  if (n == 1) {
    const V2 B0 = to_local(b0.z, b0.w, px, py, c, s);
    const V2 U0 = local_edge(a0.x, a0.y, b0.z, b0.w, c, s);
    const float de =
        edge_step<M, true>(F, A0, B0, U0, a0.z, a0.w, b0.x, b0.y, pmax, pmin, d2min);
    dlt = fminf(dlt, de);
    if (SOFT) acc.add(de, eta);
    extra_vertex<M>(F, B0, pmax, pmin, d2min);
  } else {
    V2 Acur = A0;
    float4 acur = a0, bcur = b0;
    for (int k = 0; k < n; ++k) {
      V2 Anx = A0;
      float4 anx = a0, bnx = b0;
      if (k + 1 < n) {
        anx = vt[2 * (k + 1)];
        bnx = vt[2 * (k + 1) + 1];
        Anx = to_local(anx.x, anx.y, px, py, c, s);
      }
      const V2 U = local_edge(acur.x, acur.y, anx.x, anx.y, c, s);
      const float de = edge_step<M, false>(F, Acur, Anx, U, acur.z, acur.w, bcur.x, bcur.y, pmax,
                                           pmin, d2min);
      dlt = fminf(dlt, de);
      if (SOFT) acc.add(de, eta);
      Acur = Anx;
      acur = anx;
      bcur = bnx;
    }
  }
#pragma unroll
  for (int l = 0; l < M; ++l) {
    const float2 iv = robot_interval(F, l);
    const float dl = fminf(__fsub_rn(pmax[l], iv.x), __fsub_rn(iv.y, pmin[l]));
    dlt = fminf(dlt, dl);
    if (SOFT) acc.add(dl, eta);
  }
  if (!SOFT) return synth_value(d2min, dlt, eps_sat);
  if (dlt < -eps_sat) return d2min;
  return soft_key(-acc.pen(eta));
}

// obstacle_value of the hard minimum or the soft minimum by G lanes (G
// divides 32, groups aligned): lane g of the group takes edges g, g + G, ...
// (a segment: lane 0 alone); the minima and the extreme projections are
// merged by shuffles, which are exact, so for the hard minimum every lane
// returns the serial value bit for bit.  The soft minimum accumulates its
// axes in a fixed order, so it stays serial (SOFT: lane 0 of the group
// evaluates the obstacle alone).  Every lane of the warp must call it (n = 0
// for a group without an obstacle: no loads, the value is then meaningless).
template <int M, int G, class FP>
__device__ __forceinline__ float obstacle_value_coop_hard(const FP &F, float px, float py,
                                                          float c, float s, const float4 *vt,
                                                          int n, float eps_sat, int g)
{
  float pmax[M], pmin[M];
#pragma unroll
  for (int l = 0; l < M; ++l) {
    pmax[l] = -kInf;
    pmin[l] = kInf;
  }
  float d2min = kInf, dlt = kInf;
  if (n == 1) {
    if (g == 0) {
      const float4 a0 = vt[0], b0 = vt[1];
      const V2 A0 = to_local(a0.x, a0.y, px, py, c, s);
      const V2 B0 = to_local(b0.z, b0.w, px, py, c, s);
      const V2 U0 = local_edge(a0.x, a0.y, b0.z, b0.w, c, s);
      dlt = edge_step<M, true>(F, A0, B0, U0, a0.z, a0.w, b0.x, b0.y, pmax, pmin, d2min);
      extra_vertex<M>(F, B0, pmax, pmin, d2min);
    }
  } else {
    for (int k = g; k < n; k += G) {
      const float4 ak = vt[2 * k], bk = vt[2 * k + 1];
      const float4 an = vt[2 * (k + 1 < n ? k + 1 : 0)];
      const V2 A = to_local(ak.x, ak.y, px, py, c, s);
      const V2 An = to_local(an.x, an.y, px, py, c, s);
      const V2 U = local_edge(ak.x, ak.y, an.x, an.y, c, s);
      dlt = fminf(dlt, edge_step<M, false>(F, A, An, U, ak.z, ak.w, bk.x, bk.y, pmax, pmin,
                                           d2min));
    }
  }
#pragma unroll
  for (int o = 1; o < G; o <<= 1) {
    d2min = fminf(d2min, __shfl_xor_sync(0xffffffffu, d2min, o));
    dlt = fminf(dlt, __shfl_xor_sync(0xffffffffu, dlt, o));
#pragma unroll
    for (int l = 0; l < M; ++l) {
      pmax[l] = fmaxf(pmax[l], __shfl_xor_sync(0xffffffffu, pmax[l], o));
      pmin[l] = fminf(pmin[l], __shfl_xor_sync(0xffffffffu, pmin[l], o));
    }
  }
#pragma unroll
  for (int l = 0; l < M; ++l) {
    const float2 iv = robot_interval(F, l);
    dlt = fminf(dlt, fminf(__fsub_rn(pmax[l], iv.x), __fsub_rn(iv.y, pmin[l])));
  }
  return synth_value(d2min, dlt, eps_sat);
}

template <int M, int G, bool SOFT, class FP>
__device__ __forceinline__ float obstacle_value_coop(const FP &F, float px, float py, float c,
                                                     float s, const float4 *vt, int n,
                                                     float eps_sat, float eta, int g)
{
  if constexpr (SOFT) {
    float v = kInf;
    if (g == 0 && n > 0) v = obstacle_value<M, FP, true>(F, px, py, c, s, vt, n, eps_sat, eta);
    return v;
  } else {
    return obstacle_value_coop_hard<M, G>(F, px, py, c, s, vt, n, eps_sat, g);
  }
}

// ---------------------------------------------------------------------------
// detail of one obstacle: active pair (lowest (value, pair id)) + gradient
// ---------------------------------------------------------------------------
struct Active {
  float val;      // the obstacle's min-key value (d^2, -pen, or soft_key(-pen_soft))
  float pen;      // soft penetration depth (SOFT, non-separated)
  float d2min;    // squared separation
  float dlt;      // min overlap over all axes
  bool separated;
  unsigned pid;
  int kind, l, k; // k: obstacle edge (kinds 0,1,7,8), extreme vertex (3,4), 0 (2,5,6)
  float t;        // projection parameter (kinds 0-2)
};

__device__ __forceinline__ bool better(float v, unsigned pid, float bv, unsigned bpid)
{
  return v < bv || (v == bv && pid < bpid);
}

// Running state of an obstacle's detail: per robot axis the obstacle's
// extreme projections (first vertex reaching each), the best distance and
// best obstacle-axis candidates as (value, pair id), and the minima.
template <int M>
struct DetailAcc {
  float pmax[M], pmin[M];
  int kmax[M], kmin[M];
  float d2min, dlt, bd, ba, dt;
  float d2scan;  // the scan's candidate set (far-end clamps included)
  unsigned pd, pa;
  __device__ __forceinline__ DetailAcc()
  {
#pragma unroll
    for (int l = 0; l < M; ++l) {
      pmax[l] = -kInf;
      pmin[l] = kInf;
      kmax[l] = 0;
      kmin[l] = 0;
    }
    d2min = kInf;
    d2scan = kInf;
    dlt = kInf;
    bd = kInf;
    ba = kInf;
    dt = 0.f;
    pd = PSDF_PAIR_NONE;
    pa = PSDF_PAIR_NONE;
  }
};

// Edge k of an obstacle (vt, n) into the detail state: its distance pairs
// with every robot vertex and vertex k's with every robot edge, its own
// axis, and vertex k's projections on the robot axes.
// SCAN also keeps the minimum over the scan's candidate set in q.d2scan
// (every clamped point-to-segment candidate, as edge_step takes them), with
// the same operations, so that synth_value(d2scan, dlt) is the obstacle's
// min-key value bit for bit.
template <int M, bool SOFT, bool SCAN = false>
__device__ __forceinline__ void detail_edge(const FootprintK &F, float px, float py, float c,
                                            float s, const float4 *vt, int n, int k,
                                            int orig_first, DetailAcc<M> &q, SoftAcc &acc,
                                            float eta)
{
  const bool seg = (n == 1);
  const float4 ak4 = vt[2 * k], bk4 = vt[2 * k + 1];
  float bwx, bwy;  // world B
  if (seg) {
    bwx = bk4.z;
    bwy = bk4.w;
  } else {
    const float4 an = vt[2 * (k + 1 < n ? k + 1 : 0)];
    bwx = an.x;
    bwy = an.y;
  }
  const V2 A = to_local(ak4.x, ak4.y, px, py, c, s);
  const V2 B = to_local(bwx, bwy, px, py, c, s);
  const V2 U = local_edge(ak4.x, ak4.y, bwx, bwy, c, s);
  const float ux = U.x, uy = U.y;
  const int edge = orig_first + k;
  float smin = kInf, smax = -kInf;
  int lsmin = 0, lsmax = 0;
#pragma unroll
  for (int l = 0; l < M; ++l) {
    const float wx = __fsub_rn(F.vx[l], A.x), wy = __fsub_rn(F.vy[l], A.y);
    const float t = __saturatef(__fmul_rn(__fmaf_rn(wx, ux, __fmul_rn(wy, uy)), ak4.z));
    float rx = __fmaf_rn(-t, ux, wx), ry = __fmaf_rn(-t, uy, wy);
    if (seg) {
      rx = (t == 1.0f) ? __fsub_rn(F.vx[l], B.x) : rx;
      ry = (t == 1.0f) ? __fsub_rn(F.vy[l], B.y) : ry;
    }
    const float d2 = __fmaf_rn(rx, rx, __fmul_rn(ry, ry));
    if (SCAN) q.d2scan = fminf(q.d2scan, d2);
    if (seg || t < 1.0f) {
      q.d2min = fminf(q.d2min, d2);
      const unsigned pid = make_pid(edge, kVertEdge, l);
      if (better(d2, pid, q.bd, q.pd)) { q.bd = d2; q.pd = pid; q.dt = t; }
    }
    const float sl = __fmaf_rn(wy, ux, -__fmul_rn(wx, uy));
    if (sl < smin) { smin = sl; lsmin = l; }
    if (sl > smax) { smax = sl; lsmax = l; }
    const float tp = __fmul_rn(-__fmaf_rn(wx, F.ex[l], __fmul_rn(wy, F.ey[l])), F.inv_e2[l]);
    const float qx = __fmaf_rn(tp, F.ex[l], wx), qy = __fmaf_rn(tp, F.ey[l], wy);
    const float d2p = __fmaf_rn(qx, qx, __fmul_rn(qy, qy));
    if (SCAN) {  // the clamped candidate of the scan
      const float tc = __saturatef(tp);
      const float cx = __fmaf_rn(tc, F.ex[l], wx), cy = __fmaf_rn(tc, F.ey[l], wy);
      q.d2scan = fminf(q.d2scan, __fmaf_rn(cx, cx, __fmul_rn(cy, cy)));
    }
    if (tp > 0.0f && tp < 1.0f) {
      q.d2min = fminf(q.d2min, d2p);
      const unsigned pid = make_pid(edge, kObsVRobotEdge, l);
      if (better(d2p, pid, q.bd, q.pd)) { q.bd = d2p; q.pd = pid; q.dt = tp; }
    }
    const float pr = __fmaf_rn(A.x, F.nx[l], __fmul_rn(A.y, F.ny[l]));
    if (pr > q.pmax[l]) { q.pmax[l] = pr; q.kmax[l] = k; }
    if (pr < q.pmin[l]) { q.pmin[l] = pr; q.kmin[l] = k; }
  }
  const float da = __fmaf_rn(-smin, ak4.w, bk4.y);
  const float db = __fmaf_rn(smax, ak4.w, -bk4.x);
  q.dlt = fminf(q.dlt, fminf(da, db));
  if (SOFT) acc.add(fminf(da, db), eta);
  {
    const unsigned pid = make_pid(edge, kOAxisOMax, lsmin);
    if (better(da, pid, q.ba, q.pa)) { q.ba = da; q.pa = pid; }
  }
  {
    const unsigned pid = make_pid(edge, kOAxisRMax, lsmax);
    if (better(db, pid, q.ba, q.pa)) { q.ba = db; q.pa = pid; }
  }
}

// A segment's B endpoint: its distances to the robot edges and its
// projections on the robot axes (vertex index 1).
template <int M, bool SCAN = false>
__device__ __forceinline__ void detail_seg_b(const FootprintK &F, float px, float py, float c,
                                             float s, const float4 *vt, int orig_first,
                                             DetailAcc<M> &q)
{
  const float4 b0 = vt[1];
  const V2 Bv = to_local(b0.z, b0.w, px, py, c, s);
#pragma unroll
  for (int l = 0; l < M; ++l) {
    const float wx = __fsub_rn(F.vx[l], Bv.x), wy = __fsub_rn(F.vy[l], Bv.y);
    const float tp = __fmul_rn(-__fmaf_rn(wx, F.ex[l], __fmul_rn(wy, F.ey[l])), F.inv_e2[l]);
    const float qx = __fmaf_rn(tp, F.ex[l], wx), qy = __fmaf_rn(tp, F.ey[l], wy);
    const float d2p = __fmaf_rn(qx, qx, __fmul_rn(qy, qy));
    if (SCAN) {
      const float tc = __saturatef(tp);
      const float cx = __fmaf_rn(tc, F.ex[l], wx), cy = __fmaf_rn(tc, F.ey[l], wy);
      q.d2scan = fminf(q.d2scan, __fmaf_rn(cx, cx, __fmul_rn(cy, cy)));
    }
    if (tp > 0.0f && tp < 1.0f) {
      q.d2min = fminf(q.d2min, d2p);
      const unsigned pid = make_pid(orig_first, kObsBRobotEdge, l);
      if (better(d2p, pid, q.bd, q.pd)) { q.bd = d2p; q.pd = pid; q.dt = tp; }
    }
    const float pr = __fmaf_rn(Bv.x, F.nx[l], __fmul_rn(Bv.y, F.ny[l]));
    if (pr > q.pmax[l]) { q.pmax[l] = pr; q.kmax[l] = 1; }
    if (pr < q.pmin[l]) { q.pmin[l] = pr; q.kmin[l] = 1; }
  }
}

// Robot axes, then the obstacle's value and active pair (kind, l, k and t
// re-derived from the winning pair id).
template <int M, bool SOFT>
__device__ __forceinline__ Active detail_finish(const FootprintK &F, int n, int orig_first,
                                                float eps_sat, DetailAcc<M> &q, SoftAcc &acc,
                                                float eta)
{
  const bool seg = (n == 1);
#pragma unroll
  for (int l = 0; l < M; ++l) {
    const float da = __fsub_rn(q.pmax[l], F.alo[l]);
    const float db = __fsub_rn(F.ahi[l], q.pmin[l]);
    q.dlt = fminf(q.dlt, fminf(da, db));
    if (SOFT) acc.add(fminf(da, db), eta);
    const bool bA = seg && q.kmax[l] == 1, bB = seg && q.kmin[l] == 1;
    const int eA = seg ? orig_first : orig_first + q.kmax[l];
    const int eB = seg ? orig_first : orig_first + q.kmin[l];
    const unsigned pidA = make_pid(eA, bA ? kRAxisOMaxB : kRAxisOMax, l);
    const unsigned pidB = make_pid(eB, bB ? kRAxisRMaxB : kRAxisRMax, l);
    if (better(da, pidA, q.ba, q.pa)) { q.ba = da; q.pa = pidA; }
    if (better(db, pidB, q.ba, q.pa)) { q.ba = db; q.pa = pidB; }
  }
  Active r;
  r.d2min = q.d2min;
  r.dlt = q.dlt;
  r.separated = q.dlt < -eps_sat;
  r.val = synth_value(q.d2min, q.dlt, eps_sat);
  r.pen = 0.f;
  if (SOFT && !r.separated) {
    r.pen = acc.pen(eta);
    r.val = soft_key(-r.pen);
  }
  r.pid = r.separated ? q.pd : q.pa;
  r.kind = (int)((r.pid >> kPairShiftKind) & 0xF);
  r.l = (int)(r.pid & 0xF);
  const int e = (int)(r.pid >> kPairShiftEdge) - orig_first;
  // the segment's B endpoint is vertex 1 of a robot-axis pair and vertex 0
  // (edge 0) of a robot-edge pair
  r.k = (r.kind == kRAxisOMaxB || r.kind == kRAxisRMaxB) ? 1 : e;
  r.t = r.separated ? q.dt : 0.f;
  if (r.pid == PSDF_PAIR_NONE) { r.kind = 0; r.l = 0; r.k = 0; }
  return r;
}

template <int M, bool SOFT = false>
__device__ __forceinline__ Active obstacle_detail(const FootprintK &F, float px, float py,
                                                  float c, float s, const float4 *vt, int n,
                                                  int orig_first, float eps_sat,
                                                  float eta = 0.f)
{
  SoftAcc acc;
  DetailAcc<M> q;
  for (int k = 0; k < n; ++k) detail_edge<M, SOFT>(F, px, py, c, s, vt, n, k, orig_first, q, acc, eta);
  if (n == 1) detail_seg_b<M>(F, px, py, c, s, vt, orig_first, q);
  return detail_finish<M, SOFT>(F, n, orig_first, eps_sat, q, acc, eta);
}

// The same detail by G lanes (G divides 32, groups aligned): lane g of the
// group takes edges g, g + G, ...; the states are merged by shuffles with
// the serial loop's tie rules (the lowest (value, pair id); the first vertex
// reaching an extreme projection), so every lane returns the serial
// result bit for bit.  Hard minimum only.  Every lane of the warp must call
// it (n = 0 for a lane group without an obstacle).
template <int M, int G>
__device__ __forceinline__ Active obstacle_detail_coop(const FootprintK &F, float px, float py,
                                                       float c, float s, const float4 *vt,
                                                       int n, int orig_first, float eps_sat,
                                                       int g)
{
  SoftAcc acc;
  DetailAcc<M> q;
  for (int k = g; k < n; k += G) detail_edge<M, false>(F, px, py, c, s, vt, n, k, orig_first, q, acc, 0.f);
  if (n == 1 && g == 0) detail_seg_b<M>(F, px, py, c, s, vt, orig_first, q);
#pragma unroll
  for (int o = 1; o < G; o <<= 1) {
    q.d2min = fminf(q.d2min, __shfl_xor_sync(0xffffffffu, q.d2min, o));
    q.dlt = fminf(q.dlt, __shfl_xor_sync(0xffffffffu, q.dlt, o));
    const float bd = __shfl_xor_sync(0xffffffffu, q.bd, o);
    const unsigned pd = __shfl_xor_sync(0xffffffffu, q.pd, o);
    const float dt = __shfl_xor_sync(0xffffffffu, q.dt, o);
    if (better(bd, pd, q.bd, q.pd)) { q.bd = bd; q.pd = pd; q.dt = dt; }
    const float ba = __shfl_xor_sync(0xffffffffu, q.ba, o);
    const unsigned pa = __shfl_xor_sync(0xffffffffu, q.pa, o);
    if (better(ba, pa, q.ba, q.pa)) { q.ba = ba; q.pa = pa; }
#pragma unroll
    for (int l = 0; l < M; ++l) {
      const float vmx = __shfl_xor_sync(0xffffffffu, q.pmax[l], o);
      const int kmx = __shfl_xor_sync(0xffffffffu, q.kmax[l], o);
      if (vmx > q.pmax[l] || (vmx == q.pmax[l] && kmx < q.kmax[l])) { q.pmax[l] = vmx; q.kmax[l] = kmx; }
      const float vmn = __shfl_xor_sync(0xffffffffu, q.pmin[l], o);
      const int kmn = __shfl_xor_sync(0xffffffffu, q.kmin[l], o);
      if (vmn < q.pmin[l] || (vmn == q.pmin[l] && kmn < q.kmin[l])) { q.pmin[l] = vmn; q.kmin[l] = kmn; }
    }
  }
  return detail_finish<M, false>(F, n, orig_first, eps_sat, q, acc, 0.f);
}

// obstacle_detail_coop that also returns the obstacle's min-key value as the
// scan computes it (keyval, every lane): the detail's own arithmetic plus
// the scan's unfiltered candidate minimum, so one evaluation gives both the
// key and the active pair.  Hard minimum only.
template <int M, int G>
__device__ __forceinline__ Active obstacle_scan_detail_coop(const FootprintK &F, float px,
                                                            float py, float c, float s,
                                                            const float4 *vt, int n,
                                                            int orig_first, float eps_sat,
                                                            int g, float &keyval)
{
  SoftAcc acc;
  DetailAcc<M> q;
  for (int k = g; k < n; k += G)
    detail_edge<M, false, true>(F, px, py, c, s, vt, n, k, orig_first, q, acc, 0.f);
  if (n == 1 && g == 0) detail_seg_b<M, true>(F, px, py, c, s, vt, orig_first, q);
#pragma unroll
  for (int o = 1; o < G; o <<= 1) {
    q.d2min = fminf(q.d2min, __shfl_xor_sync(0xffffffffu, q.d2min, o));
    q.d2scan = fminf(q.d2scan, __shfl_xor_sync(0xffffffffu, q.d2scan, o));
    q.dlt = fminf(q.dlt, __shfl_xor_sync(0xffffffffu, q.dlt, o));
    const float bd = __shfl_xor_sync(0xffffffffu, q.bd, o);
    const unsigned pd = __shfl_xor_sync(0xffffffffu, q.pd, o);
    const float dt = __shfl_xor_sync(0xffffffffu, q.dt, o);
    if (better(bd, pd, q.bd, q.pd)) { q.bd = bd; q.pd = pd; q.dt = dt; }
    const float ba = __shfl_xor_sync(0xffffffffu, q.ba, o);
    const unsigned pa = __shfl_xor_sync(0xffffffffu, q.pa, o);
    if (better(ba, pa, q.ba, q.pa)) { q.ba = ba; q.pa = pa; }
#pragma unroll
    for (int l = 0; l < M; ++l) {
      const float vmx = __shfl_xor_sync(0xffffffffu, q.pmax[l], o);
      const int kmx = __shfl_xor_sync(0xffffffffu, q.kmax[l], o);
      if (vmx > q.pmax[l] || (vmx == q.pmax[l] && kmx < q.kmax[l])) { q.pmax[l] = vmx; q.kmax[l] = kmx; }
      const float vmn = __shfl_xor_sync(0xffffffffu, q.pmin[l], o);
      const int kmn = __shfl_xor_sync(0xffffffffu, q.kmin[l], o);
      if (vmn < q.pmin[l] || (vmn == q.pmin[l] && kmn < q.kmin[l])) { q.pmin[l] = vmn; q.kmin[l] = kmn; }
    }
  }
  const Active a = detail_finish<M, false>(F, n, orig_first, eps_sat, q, acc, 0.f);
  keyval = synth_value(q.d2scan, a.dlt, eps_sat);
  return a;
}

// Pose gradient and edge-gradient contributions of one active pair
// (active-branch subgradient of Sec. IV-D, closed form per kind).
constexpr int kGradRows = 3;  // edge-endpoint slots an active pair touches
struct Grad {
  float gp[3];     // d sd / d (px, py, theta)
  int nrow;        // edge contributions: caller row, slot column (0 = A, 2 = B)
  int row[kGradRows], col[kGradRows];
  float gx[kGradRows], gy[kGradRows];
};

// Adds (gx, gy) to the slot of (row, col), opening one if none holds it.
// Fixed-size loops, so that the slots stay in registers.
__device__ __forceinline__ void add_row(Grad &g, int row, int col, float gx, float gy)
{
  bool merged = false;
#pragma unroll
  for (int i = 0; i < kGradRows; ++i)
    if (!merged && i < g.nrow && g.row[i] == row && g.col[i] == col) {
      g.gx[i] = __fadd_rn(g.gx[i], gx);
      g.gy[i] = __fadd_rn(g.gy[i], gy);
      merged = true;
    }
  if (merged) return;
#pragma unroll
  for (int i = 0; i < kGradRows; ++i)
    if (i == g.nrow) {
      g.row[i] = row;
      g.col[i] = col;
      g.gx[i] = gx;
      g.gy[i] = gy;
    }
  ++g.nrow;
}

// kind/l/k/t describe the active pair of obstacle (vt, n, orig_first); far
// holds the far-vertex index of each of its edges (pose-invariant).
template <int M>
__device__ Grad active_grad(const FootprintK &F, float px, float py, float c, float s,
                            const float4 *vt, const int *far, int n, int orig_first, int kind,
                            int l, int k, float t, float eps_axis)
{
  Grad g;
  g.gp[0] = g.gp[1] = g.gp[2] = 0.f;
  g.nrow = 0;
  const bool seg = (n == 1);
  // stored world endpoints of edge k (B of a polygon edge = next vertex's A)
  auto worldA = [&](int kk) { const float4 a = vt[2 * kk]; V2 r; r.x = a.x; r.y = a.y; return r; };
  auto worldB = [&](int kk) {
    V2 r;
    if (seg) { const float4 b = vt[1]; r.x = b.z; r.y = b.w; }
    else { const float4 a = vt[2 * (kk + 1 < n ? kk + 1 : 0)]; r.x = a.x; r.y = a.y; }
    return r;
  };
  // gradient of edge k's B endpoint goes to the next vertex's A slot for a
  // closed polygon, to the B slot for a segment
  auto rowB = [&](int kk) { return seg ? orig_first : orig_first + (kk + 1 < n ? kk + 1 : 0); };
  const int colB = seg ? 2 : 0;
  float vx[M], vy[M];
#pragma unroll
  for (int q = 0; q < M; ++q) { vx[q] = F.vx[q]; vy[q] = F.vy[q]; }
  float lvx = 0.f, lvy = 0.f, lex = 0.f, ley = 0.f, lnx = 0.f, lny = 0.f;
#pragma unroll
  for (int q = 0; q < M; ++q)
    if (q == l) { lvx = vx[q]; lvy = vy[q]; lex = F.ex[q]; ley = F.ey[q]; lnx = F.nx[q]; lny = F.ny[q]; }

  // every operation rounded explicitly (no contraction), so the gradient has
  // the same bits in every kernel that inlines this function
  const auto mul = [](float x, float y) { return __fmul_rn(x, y); };
  const auto add = [](float x, float y) { return __fadd_rn(x, y); };
  const auto sub = [](float x, float y) { return __fsub_rn(x, y); };
  const auto unit = [&](float rx, float ry, float &hx, float &hy) {
    // 1/|r| from the hardware reciprocal square root (a few ulp, the same
    // bits in every kernel)
    const float d2 = __fmaf_rn(rx, rx, mul(ry, ry));
    const float inv = d2 > 0.f ? rsqrtf(d2) : 0.f;
    hx = mul(rx, inv);
    hy = mul(ry, inv);
  };
  if (kind == kVertEdge) {
    const V2 Aw = worldA(k), Bw = worldB(k);
    const V2 A = to_local(Aw.x, Aw.y, px, py, c, s), B = to_local(Bw.x, Bw.y, px, py, c, s);
    const V2 U = local_edge(Aw.x, Aw.y, Bw.x, Bw.y, c, s);
    const float ux = U.x, uy = U.y;
    float rx, ry;
    if (t == 1.0f) { rx = sub(lvx, B.x); ry = sub(lvy, B.y); }
    else { rx = sub(sub(lvx, A.x), mul(t, ux)); ry = sub(sub(lvy, A.y), mul(t, uy)); }
    float hx, hy;
    unit(rx, ry, hx, hy);
    const float wx = sub(mul(c, hx), mul(s, hy)), wy = add(mul(s, hx), mul(c, hy));  // R r^
    g.gp[0] = wx; g.gp[1] = wy; g.gp[2] = sub(mul(hy, lvx), mul(hx, lvy));  // r^ . (J v)
    const float omt = sub(1.f, t);
    add_row(g, orig_first + k, 0, -mul(omt, wx), -mul(omt, wy));
    add_row(g, rowB(k), colB, -mul(t, wx), -mul(t, wy));
  } else if (kind == kObsVRobotEdge || kind == kObsBRobotEdge) {
    const V2 Xw = (kind == kObsVRobotEdge) ? worldA(k) : worldB(0);
    const V2 X = to_local(Xw.x, Xw.y, px, py, c, s);
    const float qx = __fmaf_rn(t, lex, lvx), qy = __fmaf_rn(t, ley, lvy);
    const float rx = sub(X.x, qx), ry = sub(X.y, qy);
    float hx, hy;
    unit(rx, ry, hx, hy);
    const float wx = sub(mul(c, hx), mul(s, hy)), wy = add(mul(s, hx), mul(c, hy));
    g.gp[0] = -wx; g.gp[1] = -wy; g.gp[2] = -sub(mul(hy, qx), mul(hx, qy));  // -r^ . (J q)
    if (kind == kObsVRobotEdge) add_row(g, orig_first + k, 0, wx, wy);
    else add_row(g, orig_first, 2, wx, wy);
  } else if (kind >= kRAxisOMax && kind <= kRAxisRMaxB) {
    const bool sideA = (kind == kRAxisOMax || kind == kRAxisOMaxB);
    const bool isB = (kind == kRAxisOMaxB || kind == kRAxisRMaxB);
    const V2 Xw = isB ? worldB(0) : worldA(k);
    const V2 X = to_local(Xw.x, Xw.y, px, py, c, s);
    const float Rnx = sub(mul(c, lnx), mul(s, lny)), Rny = add(mul(s, lnx), mul(c, lny));
    const float XJn = sub(mul(X.y, lnx), mul(X.x, lny));  // X . (J n), J n = (-ny, nx)
    const float gx = sideA ? Rnx : -Rnx, gy = sideA ? Rny : -Rny;
    g.gp[0] = gx; g.gp[1] = gy; g.gp[2] = sideA ? -XJn : XJn;
    if (isB) add_row(g, orig_first, 2, -gx, -gy);
    else add_row(g, orig_first + k, 0, -gx, -gy);
  } else if (kind == kOAxisOMax || kind == kOAxisRMax) {
    const bool sideA = (kind == kOAxisOMax);
    const V2 Aw = worldA(k), Bw = worldB(k);
    const float ux = sub(Bw.x, Aw.x), uy = sub(Bw.y, Aw.y);
    const float len2 = __fmaf_rn(ux, ux, mul(uy, uy));
    const float inv_len = rsqrtf(len2);  // edges are at least 1e-6 m long
    const float len = mul(len2, inv_len);
    const float gd = __fdiv_rn(1.f, add(len, eps_axis));
    const float npx = mul(-uy, gd), npy = mul(ux, gd);                          // n' (world)
    const float ntx = add(mul(c, npx), mul(s, npy)), nty = sub(mul(c, npy), mul(s, npx));  // R^T n'
    const float Rvx = sub(mul(c, lvx), mul(s, lvy)), Rvy = add(mul(s, lvx), mul(c, lvy));
    const int xk = sideA ? (seg ? 0 : far[k]) : k;  // vertex receiving d/dX
    const V2 Xw = worldA(xk);
    // delta = sgn <X - p - R v*, n'>, sd = -delta
    const float Ex = sub(sub(Xw.x, px), Rvx), Ey = sub(sub(Xw.y, py), Rvy);
    const float Dx = sideA ? Ex : -Ex, Dy = sideA ? Ey : -Ey;
    const float JvNt = sub(mul(lvx, nty), mul(lvy, ntx));  // (J v*) . R^T n'
    g.gp[0] = sideA ? npx : -npx; g.gp[1] = sideA ? npy : -npy; g.gp[2] = sideA ? JvNt : -JvNt;
    add_row(g, orig_first + xk, 0, -g.gp[0], -g.gp[1]);
    const float uhx = mul(ux, inv_len), uhy = mul(uy, inv_len);
    const float JuD = sub(mul(ux, Dy), mul(uy, Dx));
    const float gpr = -mul(gd, gd);
    // d delta / dA = -du, d delta / dB = du with du = gd J^T D + gpr u^ (J u . D)
    const float dux = add(mul(gd, Dy), mul(mul(gpr, uhx), JuD));
    const float duy = add(mul(gd, -Dx), mul(mul(gpr, uhy), JuD));
    add_row(g, orig_first + k, 0, dux, duy);
    add_row(g, rowB(k), colB, -dux, -duy);
  }
  return g;
}

// Overlap of a penetration-kind active pair (to find the flat branch of
// max(delta, 0)); same arithmetic as the scan.
template <int M>
__device__ __forceinline__ float active_overlap(const FootprintK &F, float px, float py, float c, float s,
                                const float4 *vt, int n, int kind, int l, int k)
{
  const bool seg = (n == 1);
  if (kind >= kRAxisOMax && kind <= kRAxisRMaxB) {
    const bool isB = (kind == kRAxisOMaxB || kind == kRAxisRMaxB);
    const float4 a = vt[2 * k], b = vt[1];
    const V2 X = isB ? to_local(b.z, b.w, px, py, c, s) : to_local(a.x, a.y, px, py, c, s);
    float nx = 0.f, ny = 0.f, lo = 0.f, hi = 0.f;
#pragma unroll
    for (int q = 0; q < M; ++q)
      if (q == l) { nx = F.nx[q]; ny = F.ny[q]; lo = F.alo[q]; hi = F.ahi[q]; }
    const float pr = __fmaf_rn(X.x, nx, __fmul_rn(X.y, ny));
    return (kind == kRAxisOMax || kind == kRAxisOMaxB) ? __fsub_rn(pr, lo) : __fsub_rn(hi, pr);
  }
  const float4 ak = vt[2 * k], bk = vt[2 * k + 1];
  const V2 A = to_local(ak.x, ak.y, px, py, c, s);
  float bwx = bk.z, bwy = bk.w;
  if (!seg) {
    const float4 an = vt[2 * (k + 1 < n ? k + 1 : 0)];
    bwx = an.x;
    bwy = an.y;
  }
  const V2 U = local_edge(ak.x, ak.y, bwx, bwy, c, s);
  const float ux = U.x, uy = U.y;
  float smin = kInf, smax = -kInf;
#pragma unroll
  for (int q = 0; q < M; ++q) {
    const float wx = __fsub_rn(F.vx[q], A.x), wy = __fsub_rn(F.vy[q], A.y);
    const float sl = __fmaf_rn(wy, ux, -__fmul_rn(wx, uy));
    smin = fminf(smin, sl);
    smax = fmaxf(smax, sl);
  }
  return (kind == kOAxisOMax) ? __fmaf_rn(-smin, ak.w, bk.y) : __fmaf_rn(smax, ak.w, -bk.x);
}

// Recomputes the projection parameter of a distance-kind active pair.
template <int M>
__device__ __forceinline__ float active_t(const FootprintK &F, float px, float py, float c, float s,
                          const float4 *vt, int n, int kind, int l, int k)
{
  float vx = 0.f, vy = 0.f, ex = 0.f, ey = 0.f, ie = 0.f;
#pragma unroll
  for (int q = 0; q < M; ++q)
    if (q == l) { vx = F.vx[q]; vy = F.vy[q]; ex = F.ex[q]; ey = F.ey[q]; ie = F.inv_e2[q]; }
  const bool seg = (n == 1);
  if (kind == kVertEdge) {
    const float4 ak = vt[2 * k];
    const V2 A = to_local(ak.x, ak.y, px, py, c, s);
    float bwx = vt[1].z, bwy = vt[1].w;
    if (!seg) {
      const float4 an = vt[2 * (k + 1 < n ? k + 1 : 0)];
      bwx = an.x;
      bwy = an.y;
    }
    const V2 U = local_edge(ak.x, ak.y, bwx, bwy, c, s);
    const float ux = U.x, uy = U.y;
    const float wx = __fsub_rn(vx, A.x), wy = __fsub_rn(vy, A.y);
    return __saturatef(__fmul_rn(__fmaf_rn(wx, ux, __fmul_rn(wy, uy)), ak.z));
  }
  const V2 X = (kind == kObsVRobotEdge) ? to_local(vt[2 * k].x, vt[2 * k].y, px, py, c, s)
                                        : to_local(vt[1].z, vt[1].w, px, py, c, s);
  const float wx = __fsub_rn(vx, X.x), wy = __fsub_rn(vy, X.y);
  return __fmul_rn(-__fmaf_rn(wx, ex, __fmul_rn(wy, ey)), ie);
}

// Gradient of the soft penetration (Eq. penetration_depth) of a
// non-separated obstacle: sd = -pen, d sd = sum over axes with delta > 0 of
// w_a d(-delta_a), w_a = exp(-eta (delta_a - pen)) (the softmax weights).
// Each axis contributes the closed-form gradient of its smaller side (ties by
// pair id), exactly as the active pair does in the hard case; emit(w, grad)
// is called once per contributing axis, edge axes in edge order first.
template <int M, class Emit>
__device__ __forceinline__ void soft_grad(const FootprintK &F, float px, float py, float c,
                                          float s, const float4 *vt, const int *far, int n,
                                          int orig_first, float eps_axis, float eta, float pen,
                                          Emit &&emit)
{
  const bool seg = (n == 1);
  float pmax[M], pmin[M];
  int kmax[M], kmin[M];
#pragma unroll
  for (int l = 0; l < M; ++l) {
    pmax[l] = -kInf;
    pmin[l] = kInf;
    kmax[l] = 0;
    kmin[l] = 0;
  }
  const float4 a0 = vt[0], b0 = vt[1];
  const V2 A0 = to_local(a0.x, a0.y, px, py, c, s);
  for (int k = 0; k < n; ++k) {
    const float4 ak4 = vt[2 * k], bk4 = vt[2 * k + 1];
    const V2 A = (k == 0) ? A0 : to_local(ak4.x, ak4.y, px, py, c, s);
    V2 B;
    float bwx, bwy;  // world B
    if (seg) {
      bwx = b0.z;
      bwy = b0.w;
      B = to_local(b0.z, b0.w, px, py, c, s);
    } else if (k + 1 < n) {
      const float4 an = vt[2 * (k + 1)];
      bwx = an.x;
      bwy = an.y;
      B = to_local(an.x, an.y, px, py, c, s);
    } else {
      bwx = a0.x;
      bwy = a0.y;
      B = A0;
    }
    const V2 U = local_edge(ak4.x, ak4.y, bwx, bwy, c, s);
    const float ux = U.x, uy = U.y;
    float smin = kInf, smax = -kInf;
    int lsmin = 0, lsmax = 0;
#pragma unroll
    for (int l = 0; l < M; ++l) {
      const float wx = __fsub_rn(F.vx[l], A.x), wy = __fsub_rn(F.vy[l], A.y);
      const float sl = __fmaf_rn(wy, ux, -__fmul_rn(wx, uy));
      if (sl < smin) { smin = sl; lsmin = l; }
      if (sl > smax) { smax = sl; lsmax = l; }
      const float pr = __fmaf_rn(A.x, F.nx[l], __fmul_rn(A.y, F.ny[l]));
      if (pr > pmax[l]) { pmax[l] = pr; kmax[l] = k; }
      if (pr < pmin[l]) { pmin[l] = pr; kmin[l] = k; }
    }
    const float da = __fmaf_rn(-smin, ak4.w, bk4.y);
    const float db = __fmaf_rn(smax, ak4.w, -bk4.x);
    const float dn = fminf(da, db);
    if (dn > 0.f) {
      const int edge = orig_first + k;
      const bool sideA =
          better(da, make_pid(edge, kOAxisOMax, lsmin), db, make_pid(edge, kOAxisRMax, lsmax));
      const float w = expf(__fmul_rn(-eta, __fsub_rn(dn, pen)));
      emit(w, active_grad<M>(F, px, py, c, s, vt, far, n, orig_first,
                             sideA ? kOAxisOMax : kOAxisRMax, sideA ? lsmin : lsmax, k, 0.f,
                             eps_axis));
    }
  }
  if (seg) {
    const V2 Bv = to_local(b0.z, b0.w, px, py, c, s);
#pragma unroll
    for (int l = 0; l < M; ++l) {
      const float pr = __fmaf_rn(Bv.x, F.nx[l], __fmul_rn(Bv.y, F.ny[l]));
      if (pr > pmax[l]) { pmax[l] = pr; kmax[l] = 1; }
      if (pr < pmin[l]) { pmin[l] = pr; kmin[l] = 1; }
    }
  }
#pragma unroll
  for (int l = 0; l < M; ++l) {
    const float da = __fsub_rn(pmax[l], F.alo[l]);
    const float db = __fsub_rn(F.ahi[l], pmin[l]);
    const float dn = fminf(da, db);
    if (!(dn > 0.f)) continue;
    const bool bA = seg && kmax[l] == 1, bB = seg && kmin[l] == 1;
    const int kindA = bA ? kRAxisOMaxB : kRAxisOMax, kindB = bB ? kRAxisRMaxB : kRAxisRMax;
    const int eA = seg ? orig_first : orig_first + kmax[l];
    const int eB = seg ? orig_first : orig_first + kmin[l];
    const bool sideA = better(da, make_pid(eA, kindA, l), db, make_pid(eB, kindB, l));
    const float w = expf(__fmul_rn(-eta, __fsub_rn(dn, pen)));
    emit(w, active_grad<M>(F, px, py, c, s, vt, far, n, orig_first, sideA ? kindA : kindB, l,
                           sideA ? kmax[l] : kmin[l], 0.f, eps_axis));
  }
}

// Result of the per-pose epilogue.
struct PoseOut {
  float phi;
  float g[3];  // d phi / d (x, y, theta)
  unsigned pid;
};

__device__ __forceinline__ PoseOut pose_out_failed()
{
  const float nan = __int_as_float(0x7fc00000);
  return PoseOut{nan, {nan, nan, nan}, PSDF_PAIR_NONE};
}

// Stores one pose's epilogue results; every output is optional.  stage (if
// given) receives the SQP-RTI stage parameters h = phi - d_min and
// J_g = -d phi / d x (Alg. 1).
__device__ __forceinline__ void write_pose_out(const PoseOut &r, long long p, float *phi,
                                               float *dphi, unsigned *active, float *stage,
                                               float d_min)
{
  if (phi) phi[p] = r.phi;
  if (active) active[p] = r.pid;
  if (dphi) {
    dphi[3 * p] = r.g[0];
    dphi[3 * p + 1] = r.g[1];
    dphi[3 * p + 2] = r.g[2];
  }
  if (stage) {
    reinterpret_cast<float4 *>(stage)[p] =
        make_float4(__fsub_rn(r.phi, d_min), -r.g[0], -r.g[1], -r.g[2]);
  }
}

// Value, active pair and (if want_grad) pose gradient of one pose whose
// winning obstacle o is known (none: no obstacle at all): the obstacle is
// re-evaluated with its exact candidate sets and the closed-form gradient of
// the active pair is taken (Alg. 1, value + gradient).  c, s = cos, sin of
// the pose's theta as sincosf gives them.
template <int M, bool SOFT = false>
__device__ __forceinline__ PoseOut epilogue_obstacle(const FootprintK &F, float eps_sat,
                                                     float eps_axis, float px, float py, float c,
                                                     float s, bool none, const ObsRec &o,
                                                     const float4 *__restrict__ vtx,
                                                     const int *__restrict__ far, bool want_grad,
                                                     float eta = 0.f)
{
  PoseOut r{kInf, {0.f, 0.f, 0.f}, PSDF_PAIR_NONE};
  if (none) return r;  // no obstacle at all
  const float4 *vt = vtx + 2 * (long long)o.vtx_global;
  prefetch_lines(vt, 32 * o.n);
  if (want_grad) prefetch_lines(far + o.vtx_global, 4 * o.n);
  const Active a = obstacle_detail<M, SOFT>(F, px, py, c, s, vt, o.n, o.orig_first, eps_sat, eta);
  r.pid = a.pid;
  if (SOFT && !a.separated) {
    r.phi = -a.pen;
    if (want_grad)
      soft_grad<M>(F, px, py, c, s, vt, far + o.vtx_global, o.n, o.orig_first, eps_axis, eta,
                   a.pen, [&](float w, const Grad &g) {
                     r.g[0] = __fmaf_rn(w, g.gp[0], r.g[0]);
                     r.g[1] = __fmaf_rn(w, g.gp[1], r.g[1]);
                     r.g[2] = __fmaf_rn(w, g.gp[2], r.g[2]);
                   });
    return r;
  }
  r.phi = a.separated ? sqrtf(a.val) : a.val;
  if (want_grad && (a.separated || a.dlt > 0.f)) {
    const Grad g = active_grad<M>(F, px, py, c, s, vt, far + o.vtx_global, o.n, o.orig_first,
                                  a.kind, a.l, a.k, a.t, eps_axis);
    r.g[0] = g.gp[0];
    r.g[1] = g.gp[1];
    r.g[2] = g.gp[2];
  }
  return r;
}

// The same from the pose's 64-bit min-key: row_obs is indexed by the key's
// rank (a caller row of the pose's scene).
template <int M, bool SOFT = false>
__device__ __forceinline__ PoseOut epilogue_pose(const FootprintK &F, float eps_sat,
                                                 float eps_axis, float px, float py, float theta,
                                                 unsigned long long key,
                                                 const ObsRec *__restrict__ row_obs,
                                                 const float4 *__restrict__ vtx,
                                                 const int *__restrict__ far, bool want_grad,
                                                 float eta = 0.f)
{
  if (key == ~0ull) return PoseOut{kInf, {0.f, 0.f, 0.f}, PSDF_PAIR_NONE};
  float s, c;
  sincosf(theta, &s, &c);
  const ObsRec o = row_obs[(int)(unsigned)(key & 0xffffffffu)];
  return epilogue_obstacle<M, SOFT>(F, eps_sat, eps_axis, px, py, c, s, false, o, vtx, far,
                                    want_grad, eta);
}

// epilogue_obstacle of the hard minimum by G lanes per pose (lane g of the
// group; see obstacle_detail_coop): the detail is shared out over the
// obstacle's edges, the gradient is taken by lane 0 of the group alone (the
// other lanes return it as zero).  Every lane of the warp must call it (a
// group without a pose passes none).
template <int M, int G>
__device__ __forceinline__ PoseOut epilogue_obstacle_coop(const FootprintK &F, float eps_sat,
                                                          float eps_axis, float px, float py,
                                                          float c, float s, bool none,
                                                          ObsRec o,
                                                          const float4 *__restrict__ vtx,
                                                          const int *__restrict__ far,
                                                          bool want_grad, int g,
                                                          Grad *rows = nullptr)
{
  PoseOut r{kInf, {0.f, 0.f, 0.f}, PSDF_PAIR_NONE};
  if (rows) rows->nrow = -1;  // no gradient
  if (none) o = ObsRec{0, 0, 0, 0};
  const float4 *vt = vtx + 2 * (long long)o.vtx_global;
  // the far-vertex indices the gradient reads, fetched while the detail runs
  if (want_grad && g == 0 && !none) prefetch_lines(far + o.vtx_global, 4 * o.n);
  const Active a = obstacle_detail_coop<M, G>(F, px, py, c, s, vt, o.n, o.orig_first, eps_sat, g);
  if (none) return r;
  r.pid = a.pid;
  r.phi = a.separated ? sqrtf(a.val) : a.val;
  if (want_grad && g == 0 && (a.separated || a.dlt > 0.f)) {
    const Grad gr = active_grad<M>(F, px, py, c, s, vt, far + o.vtx_global, o.n, o.orig_first,
                                   a.kind, a.l, a.k, a.t, eps_axis);
    r.g[0] = gr.gp[0];
    r.g[1] = gr.gp[1];
    r.g[2] = gr.gp[2];
    if (rows) *rows = gr;
  }
  return r;
}

// epilogue_obstacle_coop from the pose's 64-bit min-key (row_obs indexed by
// the key's rank).
template <int M, int G>
__device__ __forceinline__ PoseOut epilogue_pose_coop(const FootprintK &F, float eps_sat,
                                                      float eps_axis, float px, float py,
                                                      float theta, unsigned long long key,
                                                      const ObsRec *__restrict__ row_obs,
                                                      const float4 *__restrict__ vtx,
                                                      const int *__restrict__ far,
                                                      bool want_grad, int g,
                                                      Grad *rows = nullptr)
{
  const bool none = key == ~0ull;
  ObsRec o{0, 0, 0, 0};
  if (!none) o = row_obs[(int)(unsigned)(key & 0xffffffffu)];
  float s, c;
  sincosf(theta, &s, &c);
  return epilogue_obstacle_coop<M, G>(F, eps_sat, eps_axis, px, py, c, s, none, o, vtx, far,
                                      want_grad, g, rows);
}

// Saved backward record of one pose (psdf_saved_grad, 4 float4): the pose
// gradient of the active pair, its edge-endpoint rows (caller row * 4 +
// column, d/dx, d/dy), their count, or -1 when the pose has no gradient.
// The saved backward record of a pose (16 words) from its gradient rows.
__device__ __forceinline__ void saved_words(const Grad &g, float *w)
{
  w[0] = g.gp[0];
  w[1] = g.gp[1];
  w[2] = g.gp[2];
  w[3] = __int_as_float(g.nrow);
#pragma unroll
  for (int i = 0; i < kGradRows; ++i) {
    const bool on = i < g.nrow;
    w[4 + 3 * i] = __int_as_float(on ? 4 * g.row[i] + g.col[i] : -1);
    w[5 + 3 * i] = on ? g.gx[i] : 0.f;
    w[6 + 3 * i] = on ? g.gy[i] : 0.f;
  }
  w[13] = w[14] = w[15] = 0.f;
  if (g.nrow < 0) w[0] = w[1] = w[2] = 0.f;
}

__device__ __forceinline__ void write_saved(float4 *saved, long long p, const Grad &g)
{
  float w[16];
  saved_words(g, w);
#pragma unroll
  for (int q = 0; q < 4; ++q)
    saved[4 * p + q] = make_float4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
}

// Soft-minimum backward of one pose: when its active pair names a
// penetration axis of an obstacle that is not separated, the pose gradient
// is the softmax-weighted sum over the obstacle's axes (written to gp) and
// every axis's edge-endpoint rows go to edge(w, Grad); false otherwise (the
// hard closed form of backward_pose then applies).  row_obs / rows_total
// are those of the pose's scene.
template <int M, class Edge>
__device__ __forceinline__ bool soft_backward_pose(const FootprintK &F, float eps_sat,
                                                   float eta, float eps_axis, float px,
                                                   float py, float theta, unsigned pid,
                                                   const ObsRec *__restrict__ row_obs,
                                                   long long rows_total,
                                                   const float4 *__restrict__ vtx,
                                                   const int *__restrict__ far, float (&gp)[3],
                                                   Edge edge)
{
  const long long row = pid >> kPairShiftEdge;
  const int kind = (pid >> kPairShiftKind) & 0xF;
  if (pid == PSDF_PAIR_NONE || row >= rows_total || kind < kRAxisOMax || kind > kOAxisRMax)
    return false;
  const ObsRec o = row_obs[row];
  if (o.n == 0) return false;
  float s, c;
  sincosf(theta, &s, &c);
  const float4 *vt = vtx + 2 * (long long)o.vtx_global;
  const Active a = obstacle_detail<M, true>(F, px, py, c, s, vt, o.n, o.orig_first, eps_sat, eta);
  if (a.separated) return false;
  gp[0] = gp[1] = gp[2] = 0.f;
  soft_grad<M>(F, px, py, c, s, vt, far + o.vtx_global, o.n, o.orig_first, eps_axis, eta, a.pen,
               [&](float w, const Grad &g) {
                 gp[0] = __fmaf_rn(w, g.gp[0], gp[0]);
                 gp[1] = __fmaf_rn(w, g.gp[1], gp[1]);
                 gp[2] = __fmaf_rn(w, g.gp[2], gp[2]);
                 edge(w, g);
               });
  return true;
}

// Closed-form gradient of one pose's active pair (pid) w.r.t. the pose and
// the stored edge endpoints (rows of the pose's scene).  False when the pair
// is none, out of range, or on the flat branch of max(delta, 0).
template <int M>
__device__ __forceinline__ bool backward_pose(const FootprintK &F, float eps_axis, float px,
                                              float py, float theta, unsigned pid,
                                              const ObsRec *__restrict__ row_obs,
                                              long long rows_total,
                                              const float4 *__restrict__ vtx,
                                              const int *__restrict__ far, Grad &g)
{
  const long long row = pid >> kPairShiftEdge;
  const int kind = (pid >> kPairShiftKind) & 0xF;
  const int l = pid & 0xF;
  if (pid == PSDF_PAIR_NONE || row >= rows_total || l >= F.m || kind > kOAxisRMax) return false;
  const ObsRec o = row_obs[row];
  if (o.n == 0) return false;
  const float4 *vt = vtx + 2 * (long long)o.vtx_global;
  prefetch_lines(vt, 32 * o.n);
  prefetch_lines(far + o.vtx_global, 4 * o.n);
  int k = (int)(row - o.orig_first);
  if (kind == kObsBRobotEdge || kind == kRAxisOMaxB || kind == kRAxisRMaxB) k = 0;
  float s, c;
  sincosf(theta, &s, &c);
  float t = 0.f;
  if (kind <= kObsBRobotEdge) {
    t = active_t<M>(F, px, py, c, s, vt, o.n, kind, l, k);
  } else if (!(active_overlap<M>(F, px, py, c, s, vt, o.n, kind, l, k) > 0.f)) {
    return false;
  }
  g = active_grad<M>(F, px, py, c, s, vt, far + o.vtx_global, o.n, o.orig_first, kind, l, k, t,
                     eps_axis);
  return true;
}

}  // namespace psdf
