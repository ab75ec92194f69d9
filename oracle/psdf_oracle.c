/*
 * PSDF oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU restatement of the Polygonal Signed Distance
 * Function of "GPU-Accelerated Polygonal Signed Distance Functions for
 * Real-Time Collision Avoidance" (Sec. III-B and Sec. IV).  Only the test
 * suite, the package smoke check and the benchmark's CPU-baseline leg load
 * this library; the product path never links, imports or calls it.  It
 * shares no code, header, table or helper with the CUDA path.
 *
 * What it computes, per pose x = (p, theta) (Sec. IV-A.3, four stages):
 *   1. local frame:  A~ = R(theta)^T (A - p),  B~ = R(theta)^T (B - p)
 *   2. point-segment distances (Sec. IV-B): u = (P-A).v / (|v|^2 + eps),
 *      t = clamp(u, 0, 1), Q = A + t v, d = |P - Q|;  d_v (robot vertices to
 *      obstacle edges), d_e (obstacle vertices to robot edges), d_sep = min.
 *   3. SAT (Sec. IV-C): axes = robot outward normals and
 *      n' = rot90(u)/(|u| + eps); intervals by min/max of projections;
 *      overlap delta(n) = min(beta_i - alpha_P, beta_P - alpha_i);
 *      separated if some delta(n) < -eps_sat; penetration depth is the hard
 *      minimum of max(delta, 0) (eta <= 0) or the log-sum-exp soft minimum
 *      of Eq. (penetration_depth) (eta > 0).
 *   4. synthesis (Sec. IV-D): sd_i = d_sep if separated else -pen;
 *      phi = min_i sd_i (Eq. psdf_value).
 * The gradient is the active-branch subgradient of Sec. IV-D, written in
 * closed form per active feature (the "active pair, margins, gradients"
 * block of eval_obstacle).
 *
 * Readings taken where the paper is silent (each restated in the design
 * notes of the repository):
 *   R1  A single-edge obstacle (a LiDAR segment) keeps both endpoints in
 *       its vertex set, so its sd is the exact polygon-to-segment distance.
 *   R2  For closed polygons a vertex-to-edge candidate whose clamp lands on
 *       the far endpoint (t == 1) is not a separate candidate: it is the
 *       next edge's start vertex, already a candidate of that edge.  An
 *       obstacle-vertex-to-robot-edge candidate counts only for interior
 *       projections (0 < t < 1); its endpoints are robot vertices, covered
 *       by the vertex-to-edge pool.  The minimum value is unchanged; the
 *       choice of active pair becomes unique at vertex-vertex contacts.
 *   R3  Active pair id = (edge << 8) | (kind << 4) | l, ties broken by the
 *       lowest (value, id); across obstacles by the lowest obstacle index.
 *   R4  On an obstacle's own edge normal the obstacle interval is attained
 *       along the edge itself; the gradient is attributed to that edge's
 *       stored A entry (lower side), or, for a closed polygon, to the
 *       farthest vertex (upper side; for a segment both sides use A).
 *   R5  With no obstacle at all phi = +inf, pair = 0xFFFFFFFF, grad = 0.
 *   R6  A closed polygon's vertex is stored twice (A of its edge, B of the
 *       previous edge).  The derivative with respect to one stored copy alone
 *       has a kink wherever the vertex lies on an edge line (always, on the
 *       polygon's own edge normals), so gradients are taken with respect to
 *       the vertex (both copies moved together) and reported in its A slot;
 *       the B slots of closed polygons receive zero.  A segment's A and B are
 *       distinct points and keep their own gradients.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PID_NONE 0xFFFFFFFFu
#define PID(edge, kind, l) (((unsigned)(edge) << 8) | ((unsigned)(kind) << 4) | (unsigned)(l))

/* kinds of active pairs */
enum {
  K_VERT_EDGE = 0,   /* robot vertex l -> obstacle edge e                    */
  K_OBSV_REDGE = 1,  /* obstacle vertex A_e -> interior of robot edge l      */
  K_OBSB_REDGE = 2,  /* segment endpoint B_e -> interior of robot edge l     */
  K_RAX_OMAX = 3,    /* robot axis l, delta = beta_i - alpha_P, extreme A_e  */
  K_RAX_RMAX = 4,    /* robot axis l, delta = beta_P - alpha_i, extreme A_e  */
  K_RAX_OMAX_B = 5,  /* as 3, extreme vertex is a segment's B_e              */
  K_RAX_RMAX_B = 6,  /* as 4, extreme vertex is a segment's B_e              */
  K_OAX_OMAX = 7,    /* obstacle axis of edge e, delta = beta_i - alpha_P,
                        robot extreme vertex l (the robot minimum)          */
  K_OAX_RMAX = 8     /* obstacle axis of edge e, delta = beta_P - alpha_i,
                        robot extreme vertex l (the robot maximum)          */
};

typedef struct {
  double eps_seg;  /* epsilon of the projection factor u (Sec. IV-B)        */
  double eps_axis; /* epsilon of the obstacle-axis normalisation (Sec. IV-C) */
  double eps_sat;  /* separating-axis tolerance (Sec. IV-C)                  */
  double eta;      /* soft-min sharpness; <= 0 selects the hard minimum      */
} oracle_params;

typedef struct {
  const double *fp;    /* [m][2] robot footprint, CCW, local frame */
  int m;
  const double *edges; /* [E][4] Ax Ay Bx By, world frame          */
  const int *offs;     /* [M+1]                                    */
  int M;
  oracle_params prm;
  double re[16][2];    /* robot edge vectors e_l = v_{l+1} - v_l    */
  double rn[16][2];    /* robot outward unit normals n_l            */
} Ctx;

/* one distance candidate (Sec. IV-B) */
typedef struct {
  double v;      /* squared distance */
  unsigned pid;
  int kind, l, k; /* l: robot vertex / edge, k: obstacle edge or vertex   */
  double t;       /* clamped projection parameter                          */
} DCand;

/* one SAT candidate: one side of one axis (Sec. IV-C) */
typedef struct {
  double v;       /* delta side value */
  unsigned pid;
  int kind, l, k; /* l: robot axis or robot extreme vertex; k: obstacle
                     axis edge or obstacle extreme vertex (index into W) */
  int axis;       /* 0..m-1 robot axes, m + j obstacle axis j            */
  double vgap;    /* margin of the extreme-vertex choice (pair id)        */
  double egap;    /* margin of the vertex that receives the edge gradient */
} ACand;

typedef struct {
  double sd;
  int separated;
  unsigned pid;
  double gap;   /* pair-id margin within the obstacle (metres)            */
  double egap;  /* margin of the edge-gradient attribution                */
  unsigned twin;
  double g[3];  /* d sd / d (px, py, theta)                               */
} ObsOut;

static double dot2(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1]; }

/* world -> robot-local frame: R(theta)^T (X - p) (Sec. IV-A.3, stage 1) */
static void to_local(double c, double s, double px, double py, double X, double Y, double *out)
{
  double dx = X - px, dy = Y - py;
  out[0] = c * dx + s * dy;
  out[1] = -s * dx + c * dy;
}

/* R(theta) v */
static void rot(double c, double s, const double *v, double *out)
{
  out[0] = c * v[0] - s * v[1];
  out[1] = s * v[0] + c * v[1];
}

/* J v with J = [[0,-1],[1,0]] (d R / d theta = R J) */
static void jmul(const double *v, double *out)
{
  out[0] = -v[1];
  out[1] = v[0];
}

/* add (gx, gy) to the gradient of edge j's B endpoint: for a closed polygon
   that point is vertex j+1, reported in the A slot of edge j+1 (R6) */
static void add_grad_B(double *gedge, int j, int n, int seg, double gx, double gy)
{
  int row = seg ? j : (j + 1) % n;
  int col = seg ? 2 : 0;
  gedge[4 * row + col] += gx;
  gedge[4 * row + col + 1] += gy;
}

static void ctx_init(Ctx *C, const double *fp, int m, const double *edges, const int *offs,
                     int M, const oracle_params *prm)
{
  C->fp = fp; C->m = m; C->edges = edges; C->offs = offs; C->M = M; C->prm = *prm;
  for (int l = 0; l < m; ++l) {
    const double *a = fp + 2 * l, *b = fp + 2 * ((l + 1) % m);
    double ex = b[0] - a[0], ey = b[1] - a[1];
    double len = sqrt(ex * ex + ey * ey);
    C->re[l][0] = ex; C->re[l][1] = ey;
    /* outward normal of a CCW polygon: rotate the edge by -90 degrees */
    C->rn[l][0] = ey / len; C->rn[l][1] = -ex / len;
  }
}

/*
 * Evaluate obstacle i at one pose.  detail == 0: only sd / separated.
 * detail == 1: also the active pair, margins and gradients; gedge (if not
 * NULL) receives d sd / d stored edge rows [n][4] of this obstacle.
 */
static void eval_obstacle(const Ctx *C, int i, const double *pose, int detail, ObsOut *out,
                          double *gedge)
{
  const int m = C->m;
  const int e0 = C->offs[i];
  const int n = C->offs[i + 1] - e0;
  const int seg = (n == 1);
  const double px = pose[0], py = pose[1], th = pose[2];
  const double c = cos(th), s = sin(th);
  const oracle_params *P = &C->prm;

  /* Stage 1: transform stored endpoints into the robot frame */
  double *At = (double *)malloc(sizeof(double) * 2 * (size_t)n);
  double *Bt = (double *)malloc(sizeof(double) * 2 * (size_t)n);
  for (int j = 0; j < n; ++j) {
    const double *E = C->edges + 4 * (size_t)(e0 + j);
    to_local(c, s, px, py, E[0], E[1], At + 2 * j);
    to_local(c, s, px, py, E[2], E[3], Bt + 2 * j);
  }
  /* obstacle vertex set V_obs (Eq. obstacle_vertex_set; R1 for segments) */
  const int nw = seg ? 2 : n;
  double W[2 * 4096 + 4];
  int nwc = nw > 4096 ? 4096 : nw;
  for (int k = 0; k < nwc; ++k) {
    const double *src = (seg && k == 1) ? Bt : At + 2 * k;
    W[2 * k] = src[0]; W[2 * k + 1] = src[1];
  }

  /* ---------------- Stage 2: point-segment distance pools ------------- */
  size_t capd = (size_t)n * m * 2 + 2 * (size_t)m + 8;
  DCand *dc = detail ? (DCand *)malloc(sizeof(DCand) * capd) : NULL;
  size_t nd = 0;
  double dmin2 = INFINITY;

  /* d_v: robot vertex l to obstacle edge j (eq. d_v) */
  for (int j = 0; j < n; ++j) {
    double v[2] = {Bt[2 * j] - At[2 * j], Bt[2 * j + 1] - At[2 * j + 1]};
    double vv = dot2(v, v);
    for (int l = 0; l < m; ++l) {
      const double *V0 = C->fp + 2 * l;
      double w[2] = {V0[0] - At[2 * j], V0[1] - At[2 * j + 1]};
      double u = dot2(w, v) / (vv + P->eps_seg);
      double t = u < 0.0 ? 0.0 : (u > 1.0 ? 1.0 : u);
      if (!seg && t == 1.0) continue; /* R2: the next edge's start vertex */
      double r[2];
      if (t == 1.0) { r[0] = V0[0] - Bt[2 * j]; r[1] = V0[1] - Bt[2 * j + 1]; }
      else { r[0] = w[0] - t * v[0]; r[1] = w[1] - t * v[1]; }
      double d2 = dot2(r, r);
      if (d2 < dmin2) dmin2 = d2;
      if (detail) { DCand q = {d2, PID(e0 + j, K_VERT_EDGE, l), K_VERT_EDGE, l, j, t}; dc[nd++] = q; }
    }
  }
  /* d_e: obstacle vertex w to robot edge l (eq. d_e), interior projections (R2) */
  for (int k = 0; k < nw; ++k) {
    const double *w0 = W + 2 * k;
    for (int l = 0; l < m; ++l) {
      const double *V0 = C->fp + 2 * l;
      const double *e = C->re[l];
      double w[2] = {w0[0] - V0[0], w0[1] - V0[1]};
      double u = dot2(w, e) / (dot2(e, e) + P->eps_seg);
      double t = u < 0.0 ? 0.0 : (u > 1.0 ? 1.0 : u);
      if (t <= 0.0 || t >= 1.0) continue;
      double r[2] = {w[0] - t * e[0], w[1] - t * e[1]};
      double d2 = dot2(r, r);
      if (d2 < dmin2) dmin2 = d2;
      if (detail) {
        int kind = (seg && k == 1) ? K_OBSB_REDGE : K_OBSV_REDGE;
        int edge = seg ? e0 : e0 + k;
        DCand q = {d2, PID(edge, kind, l), kind, l, k, t};
        dc[nd++] = q;
      }
    }
  }

  /* ---------------- Stage 3: SAT -------------------------------------- */
  const int naxes = m + n;
  ACand *ac = detail ? (ACand *)malloc(sizeof(ACand) * 2 * (size_t)naxes) : NULL;
  double *axd = (double *)malloc(sizeof(double) * (size_t)naxes); /* delta(n) */
  size_t na = 0;
  double delta_min = INFINITY;

  /* robot axes n_l */
  for (int l = 0; l < m; ++l) {
    const double *nl = C->rn[l];
    double aP = INFINITY, bP = -INFINITY;
    for (int q = 0; q < m; ++q) {
      double pr = dot2(C->fp + 2 * q, nl);
      if (pr < aP) aP = pr;
      if (pr > bP) bP = pr;
    }
    double ai = INFINITY, bi = -INFINITY;
    int kmin = 0, kmax = 0;
    for (int k = 0; k < nw; ++k) {
      double pr = dot2(W + 2 * k, nl);
      if (pr < ai) { ai = pr; kmin = k; }
      if (pr > bi) { bi = pr; kmax = k; }
    }
    double da = bi - aP, db = bP - ai;
    double dn = da < db ? da : db;
    axd[l] = dn;
    if (dn < delta_min) delta_min = dn;
    if (detail) {
      /* margins of the extreme obstacle vertices */
      double g2max = INFINITY, g2min = INFINITY;
      for (int k = 0; k < nw; ++k) {
        double pr = dot2(W + 2 * k, nl);
        if (k != kmax && bi - pr < g2max) g2max = bi - pr;
        if (k != kmin && pr - ai < g2min) g2min = pr - ai;
      }
      int kA = (seg && kmax == 1) ? K_RAX_OMAX_B : K_RAX_OMAX;
      int kB = (seg && kmin == 1) ? K_RAX_RMAX_B : K_RAX_RMAX;
      int edA = seg ? e0 : e0 + kmax, edB = seg ? e0 : e0 + kmin;
      ACand a1 = {da, PID(edA, kA, l), kA, l, kmax, l, g2max, g2max};
      ACand a2 = {db, PID(edB, kB, l), kB, l, kmin, l, g2min, g2min};
      ac[na++] = a1;
      ac[na++] = a2;
    }
  }
  /* obstacle axes n'_j = rot90(u)/(|u| + eps) */
  for (int j = 0; j < n; ++j) {
    double u[2] = {Bt[2 * j] - At[2 * j], Bt[2 * j + 1] - At[2 * j + 1]};
    double un = sqrt(dot2(u, u)) + P->eps_axis;
    double nj[2] = {-u[1] / un, u[0] / un};
    double aP = INFINITY, bP = -INFINITY;
    int lmin = 0, lmax = 0;
    for (int q = 0; q < m; ++q) {
      double pr = dot2(C->fp + 2 * q, nj);
      if (pr < aP) { aP = pr; lmin = q; }
      if (pr > bP) { bP = pr; lmax = q; }
    }
    double ai = INFINITY, bi = -INFINITY;
    int kmax = 0;
    for (int k = 0; k < nw; ++k) {
      double pr = dot2(W + 2 * k, nj);
      if (pr < ai) ai = pr;
      if (pr > bi) { bi = pr; kmax = k; }
    }
    double da = bi - aP, db = bP - ai;
    double dn = da < db ? da : db;
    axd[m + j] = dn;
    if (dn < delta_min) delta_min = dn;
    if (detail) {
      double g2min = INFINITY, g2max = INFINITY, gfar = INFINITY;
      for (int q = 0; q < m; ++q) {
        double pr = dot2(C->fp + 2 * q, nj);
        if (q != lmin && pr - aP < g2min) g2min = pr - aP;
        if (q != lmax && bP - pr < g2max) g2max = bP - pr;
      }
      /* R4: the upper end of the obstacle interval is attained at the far
         vertex (closed polygon) or along the segment itself (use A) */
      int kfar = seg ? 0 : kmax;
      if (!seg)
        for (int k = 0; k < nw; ++k) {
          double pr = dot2(W + 2 * k, nj);
          if (k != kmax && bi - pr < gfar) gfar = bi - pr;
        }
      ACand a1 = {da, PID(e0 + j, K_OAX_OMAX, lmin), K_OAX_OMAX, lmin, kfar, m + j, g2min,
                  g2min < gfar ? g2min : gfar};
      ACand a2 = {db, PID(e0 + j, K_OAX_RMAX, lmax), K_OAX_RMAX, lmax, j, m + j, g2max, g2max};
      ac[na++] = a1;
      ac[na++] = a2;
    }
  }

  /* separated test (Sec. IV-C) */
  int separated = 0;
  for (int a = 0; a < naxes; ++a)
    if (axd[a] < -P->eps_sat) { separated = 1; break; }

  /* ---------------- Stage 4: synthesis (Sec. IV-D) -------------------- */
  double sd;
  double pen_soft = 0.0;
  if (separated) {
    sd = sqrt(dmin2);
  } else if (P->eta <= 0.0) {
    double pen = delta_min > 0.0 ? delta_min : 0.0; /* min_n max(delta, 0) */
    sd = -pen;
  } else {
    /* Eq. (penetration_depth): -(1/eta) log sum exp(-eta * delta_+) */
    double mu = INFINITY;
    for (int a = 0; a < naxes; ++a) {
      double dp = axd[a] > 0.0 ? axd[a] : 0.0;
      if (dp < mu) mu = dp;
    }
    double ssum = 0.0;
    for (int a = 0; a < naxes; ++a) {
      double dp = axd[a] > 0.0 ? axd[a] : 0.0;
      ssum += exp(-P->eta * (dp - mu));
    }
    pen_soft = mu - log(ssum) / P->eta;
    sd = -pen_soft;
  }
  out->sd = sd;
  out->separated = separated;

  if (!detail) {
    free(At); free(Bt); free(axd);
    return;
  }

  /* ---------------- active pair, margins, gradients -------------------- */
  out->twin = PID_NONE;
  out->g[0] = out->g[1] = out->g[2] = 0.0;
  out->egap = INFINITY;
  if (gedge) memset(gedge, 0, sizeof(double) * 4 * (size_t)n);

  if (separated) {
    size_t b = 0;
    for (size_t q = 1; q < nd; ++q)
      if (dc[q].v < dc[b].v || (dc[q].v == dc[b].v && dc[q].pid < dc[b].pid)) b = q;
    double dbest = sqrt(dc[b].v);
    double gap = INFINITY;
    for (size_t q = 0; q < nd; ++q)
      if (q != b) {
        double gq = sqrt(dc[q].v) - dbest;
        if (gq < gap) gap = gq;
      }
    /* distance from the SAT decision (delta_min < 0 here) */
    if (-delta_min < gap) gap = -delta_min;
    out->pid = dc[b].pid;
    out->gap = gap;
    out->egap = gap;
    const DCand *a = &dc[b];
    double d = dbest;
    if (a->kind == K_VERT_EDGE) {
      /* r = v_l - Q~ ; d/dp = R r^, d/dtheta = r^ . (J v_l) */
      const double *V0 = C->fp + 2 * a->l;
      int j = a->k;
      double r[2];
      if (a->t == 1.0) { r[0] = V0[0] - Bt[2 * j]; r[1] = V0[1] - Bt[2 * j + 1]; }
      else {
        double v[2] = {Bt[2 * j] - At[2 * j], Bt[2 * j + 1] - At[2 * j + 1]};
        r[0] = V0[0] - At[2 * j] - a->t * v[0];
        r[1] = V0[1] - At[2 * j + 1] - a->t * v[1];
      }
      double rh[2] = {0.0, 0.0};
      if (d > 0.0) { rh[0] = r[0] / d; rh[1] = r[1] / d; }
      double wr[2], jv[2];
      rot(c, s, rh, wr);
      jmul(V0, jv);
      out->g[0] = wr[0]; out->g[1] = wr[1]; out->g[2] = dot2(rh, jv);
      if (gedge) {
        /* envelope theorem: d/dA = -(1-t) R r^, d/dB = -t R r^ */
        gedge[4 * j + 0] -= (1.0 - a->t) * wr[0];
        gedge[4 * j + 1] -= (1.0 - a->t) * wr[1];
        add_grad_B(gedge, j, n, seg, -a->t * wr[0], -a->t * wr[1]);
      }
    } else {
      /* r' = w - q, q = v_l + t e_l ; d/dp = -R r^', d/dtheta = -r^'.(J q) */
      const double *V0 = C->fp + 2 * a->l;
      const double *e = C->re[a->l];
      const double *w0 = W + 2 * a->k;
      double q[2] = {V0[0] + a->t * e[0], V0[1] + a->t * e[1]};
      double r[2] = {w0[0] - q[0], w0[1] - q[1]};
      double rh[2] = {0.0, 0.0};
      if (d > 0.0) { rh[0] = r[0] / d; rh[1] = r[1] / d; }
      double wr[2], jq[2];
      rot(c, s, rh, wr);
      jmul(q, jq);
      out->g[0] = -wr[0]; out->g[1] = -wr[1]; out->g[2] = -dot2(rh, jq);
      if (gedge) {
        int row = seg ? 0 : a->k;
        int col = (a->kind == K_OBSB_REDGE) ? 2 : 0;
        gedge[4 * row + col] += wr[0];
        gedge[4 * row + col + 1] += wr[1];
      }
    }
  } else {
    size_t b = 0;
    for (size_t q = 1; q < na; ++q)
      if (ac[q].v < ac[b].v || (ac[q].v == ac[b].v && ac[q].pid < ac[b].pid)) b = q;
    const ACand *best = &ac[b];
    /* twin axes: exactly antiparallel robot normals, or obstacle normals of
       the same obstacle antiparallel within 1e-6 rad; the twin's opposite
       side carries the same overlap */
    double gap = INFINITY;
    for (size_t q = 0; q < na; ++q) {
      if (q == b) continue;
      const ACand *o = &ac[q];
      int twin = 0;
      int opp_side = 0;
      if (best->axis < m && o->axis < m) {
        const double *n1 = C->rn[best->axis], *n2 = C->rn[o->axis];
        opp_side = ((best->kind == K_RAX_OMAX || best->kind == K_RAX_OMAX_B) !=
                    (o->kind == K_RAX_OMAX || o->kind == K_RAX_OMAX_B));
        if (opp_side && n1[0] == -n2[0] && n1[1] == -n2[1]) twin = 1;
      } else if (best->axis >= m && o->axis >= m && best->axis != o->axis) {
        int j1 = best->axis - m, j2 = o->axis - m;
        double u1[2] = {Bt[2 * j1] - At[2 * j1], Bt[2 * j1 + 1] - At[2 * j1 + 1]};
        double u2[2] = {Bt[2 * j2] - At[2 * j2], Bt[2 * j2 + 1] - At[2 * j2 + 1]};
        double l1 = sqrt(dot2(u1, u1)), l2 = sqrt(dot2(u2, u2));
        double cr = (u1[0] * u2[1] - u1[1] * u2[0]) / (l1 * l2);
        double dt = dot2(u1, u2) / (l1 * l2);
        opp_side = (best->kind != o->kind);
        if (opp_side && dt < 0.0 && fabs(cr) < 1e-6) {
          twin = 1;
          if (out->twin == PID_NONE || o->pid < out->twin) out->twin = o->pid;
        }
      }
      if (twin) continue;
      double gq = o->v - best->v;
      if (gq < gap) gap = gq;
    }
    if (best->vgap < gap) gap = best->vgap;
    double dpos = best->v;
    if (fabs(dpos) < gap) gap = fabs(dpos); /* distance from the SAT switch */
    out->pid = best->pid;
    out->gap = gap;
    out->egap = best->egap < gap ? best->egap : gap;
    if (out->twin != PID_NONE) out->egap = 0.0; /* attribution depends on rounding */

    /* hard or soft gradient: sd = -pen.  For the hard minimum one axis is
       active; the soft minimum weights every axis with delta > 0 by the
       softmax of -eta * delta_+ (derivative of Eq. penetration_depth). */
    int nact = 0;
    for (int a = 0; a < naxes; ++a) {
      double wgt;
      int side_is_a;
      int ka, kl;
      if (P->eta <= 0.0) {
        if (a != best->axis) continue;
        wgt = 1.0;
        if (delta_min <= 0.0) wgt = 0.0; /* pen = max(delta,0) at 0: flat branch */
        side_is_a = (best->kind == K_RAX_OMAX || best->kind == K_RAX_OMAX_B ||
                     best->kind == K_OAX_OMAX);
        ka = best->k; kl = best->l;
      } else {
        if (!(axd[a] > 0.0)) continue;
        /* weight = exp(-eta (delta_a - pen_soft)) = softmax of -eta delta_+ */
        wgt = exp(-P->eta * (axd[a] - pen_soft));
        /* the active side of this axis: the smaller of its two candidates */
        const ACand *s1 = &ac[2 * a], *s2 = &ac[2 * a + 1];
        const ACand *sa = (s1->v < s2->v || (s1->v == s2->v && s1->pid < s2->pid)) ? s1 : s2;
        side_is_a = (sa->kind == K_RAX_OMAX || sa->kind == K_RAX_OMAX_B || sa->kind == K_OAX_OMAX);
        ka = sa->k; kl = sa->l;
      }
      ++nact;
      double gp[3];
      double ge_row_k[4] = {0, 0, 0, 0}; int row_k = -1, col_k = 0;
      double ge_u[2] = {0, 0}; int row_u = -1;
      if (a < m) {
        /* robot axis n_l, extreme obstacle vertex W_k.
           side a: sd = -(<W_k,n> - alpha_P):  d/dp = R n, d/dtheta = -W_k.(J n), d/dX_k = -R n
           side b: sd = <W_k,n> - beta_P:      all signs flipped                              */
        const double *nl = C->rn[a];
        double Rn[2], Jn[2];
        rot(c, s, nl, Rn);
        jmul(nl, Jn);
        double sg = side_is_a ? 1.0 : -1.0;
        const double *Wk = W + 2 * ka;
        gp[0] = sg * Rn[0]; gp[1] = sg * Rn[1]; gp[2] = -sg * dot2(Wk, Jn);
        row_k = seg ? 0 : ka; col_k = (seg && ka == 1) ? 2 : 0;
        ge_row_k[0] = -sg * Rn[0]; ge_row_k[1] = -sg * Rn[1];
      } else {
        /* obstacle axis of edge j: n' = J u / (|u| + eps) in the world frame.
           side a: delta = <X_far - p - R v*, n'>,  side b: delta = <R v* + p - X_j, n'> */
        int j = a - m;
        const double *E = C->edges + 4 * (size_t)(e0 + j);
        double u[2] = {E[2] - E[0], E[3] - E[1]};
        double ul = sqrt(dot2(u, u));
        double gden = 1.0 / (ul + P->eps_axis);
        double np[2] = {-u[1] * gden, u[0] * gden};
        double nt[2] = {c * np[0] + s * np[1], -s * np[0] + c * np[1]}; /* R^T n' */
        const double *vs = C->fp + 2 * kl;
        double Rv[2], Jv[2];
        rot(c, s, vs, Rv);
        jmul(vs, Jv);
        double Xw[2];
        int xrow;
        if (side_is_a) {
          /* far vertex: stored A of edge ka (polygon) or the segment's A */
          xrow = seg ? 0 : ka;
        } else {
          xrow = j;
        }
        const double *EX = C->edges + 4 * (size_t)(e0 + xrow);
        Xw[0] = EX[0]; Xw[1] = EX[1];
        double D[2];
        double sgn = side_is_a ? 1.0 : -1.0; /* delta = sgn * <X - p - R v*, n'> */
        D[0] = sgn * (Xw[0] - pose[0] - Rv[0]);
        D[1] = sgn * (Xw[1] - pose[1] - Rv[1]);
        /* d delta / d p = -sgn n', d delta / d theta = -sgn (J v*).n~ ,
           d delta / d X = sgn n', d delta / d u = g J^T D + g' u^ <J u, D> */
        double ddp[2] = {-sgn * np[0], -sgn * np[1]};
        double ddth = -sgn * dot2(Jv, nt);
        double ddX[2] = {sgn * np[0], sgn * np[1]};
        double uh[2] = {u[0] / ul, u[1] / ul};
        double JtD[2] = {D[1], -D[0]};
        double Ju[2] = {-u[1], u[0]};
        double gpr = -gden * gden;
        double JuD = dot2(Ju, D);
        double ddu[2] = {gden * JtD[0] + gpr * uh[0] * JuD, gden * JtD[1] + gpr * uh[1] * JuD};
        /* sd = -delta */
        gp[0] = -ddp[0]; gp[1] = -ddp[1]; gp[2] = -ddth;
        row_k = xrow; col_k = 0;
        ge_row_k[0] = -ddX[0]; ge_row_k[1] = -ddX[1];
        row_u = j;
        ge_u[0] = -ddu[0]; ge_u[1] = -ddu[1];
      }
      out->g[0] += wgt * gp[0];
      out->g[1] += wgt * gp[1];
      out->g[2] += wgt * gp[2];
      if (gedge) {
        if (row_k >= 0) {
          gedge[4 * row_k + col_k] += wgt * ge_row_k[0];
          gedge[4 * row_k + col_k + 1] += wgt * ge_row_k[1];
        }
        if (row_u >= 0) {
          /* u = B - A */
          gedge[4 * row_u + 0] -= wgt * ge_u[0];
          gedge[4 * row_u + 1] -= wgt * ge_u[1];
          add_grad_B(gedge, row_u, n, seg, wgt * ge_u[0], wgt * ge_u[1]);
        }
      }
    }
    (void)nact;
  }

  free(At); free(Bt); free(axd);
  free(dc); free(ac);
}

typedef struct {
  double phi;
  unsigned pid;
  double g[3];
  double margin;
  double egap;
  unsigned twin;
  int obstacle;
} PoseOut;

static void eval_pose(const Ctx *C, const double *pose, PoseOut *o, double *gedge_scratch)
{
  int best = -1;
  double bsd = INFINITY;
  double *sdv = (double *)malloc(sizeof(double) * (size_t)(C->M > 0 ? C->M : 1));
  for (int i = 0; i < C->M; ++i) {
    ObsOut ob;
    eval_obstacle(C, i, pose, 0, &ob, NULL);
    sdv[i] = ob.sd;
    if (best < 0 || ob.sd < bsd) { best = i; bsd = ob.sd; }
  }
  /* runner-up obstacle: 'second' skips exact ties (obstacles sharing the
     active vertex resolve by index on both sides of a comparison),
     'second_tied' does not (it bounds the edge-gradient attribution) */
  double second = INFINITY, second_tied = INFINITY;
  for (int i = 0; i < C->M; ++i) {
    if (i == best) continue;
    if (sdv[i] < second_tied) second_tied = sdv[i];
    if (sdv[i] != bsd && sdv[i] < second) second = sdv[i];
  }
  free(sdv);
  o->obstacle = best;
  if (best < 0) {
    o->phi = INFINITY; o->pid = PID_NONE; o->g[0] = o->g[1] = o->g[2] = 0.0;
    o->margin = INFINITY; o->egap = INFINITY; o->twin = PID_NONE;
    return;
  }
  ObsOut ob;
  eval_obstacle(C, best, pose, 1, &ob, gedge_scratch);
  o->phi = ob.sd;
  o->pid = ob.pid;
  o->g[0] = ob.g[0]; o->g[1] = ob.g[1]; o->g[2] = ob.g[2];
  double mg = ob.gap;
  if (second - bsd < mg) mg = second - bsd;
  o->margin = mg;
  o->egap = ob.egap < mg ? ob.egap : mg;
  if (second_tied - bsd < o->egap) o->egap = second_tied - bsd;
  o->twin = ob.twin;
}

static int max_obstacle_edges(const int *offs, int M)
{
  int mx = 1;
  for (int i = 0; i < M; ++i)
    if (offs[i + 1] - offs[i] > mx) mx = offs[i + 1] - offs[i];
  return mx;
}

static int check_inputs(int m, const int *offs, int M)
{
  if (m < 3 || m > 16 || M < 0) return -1;
  for (int i = 0; i < M; ++i) {
    int n = offs[i + 1] - offs[i];
    if (n != 1 && n < 3) return -2;
    if (n > 4096) return -3;
  }
  return 0;
}

/*
 * phi[P], pair[P], dphi[P][3] (d phi / d (px, py, theta)), margin[P]
 * (distance of the active choice from a tie, metres), egap[P] (margin of
 * the edge-gradient attribution), twin[P] (pair id of an antiparallel twin
 * axis that carries the same overlap, or 0xFFFFFFFF).  Any output pointer
 * may be NULL.  Returns 0, or a negative code on invalid sizes.
 */
int oracle_psdf_eval(const double *footprint, int m, const double *edges, const int *offsets,
                     int M, const double *poses, long P, const oracle_params *prm, double *phi,
                     unsigned *pair, double *dphi, double *margin, double *egap, unsigned *twin,
                     int nthreads)
{
  int rc = check_inputs(m, offsets, M);
  if (rc) return rc;
  Ctx C;
  ctx_init(&C, footprint, m, edges, offsets, M, prm);
  int mx = max_obstacle_edges(offsets, M);
  (void)mx;
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads)
#endif
  for (long q = 0; q < P; ++q) {
    PoseOut o;
    eval_pose(&C, poses + 3 * q, &o, NULL);
    if (phi) phi[q] = o.phi;
    if (pair) pair[q] = o.pid;
    if (dphi) { dphi[3 * q] = o.g[0]; dphi[3 * q + 1] = o.g[1]; dphi[3 * q + 2] = o.g[2]; }
    if (margin) margin[q] = o.margin;
    if (egap) egap[q] = o.egap;
    if (twin) twin[q] = o.twin;
  }
  (void)nthreads;
  return 0;
}

/*
 * Backward of phi (Alg. 1, PSDF_Backward): grad_pose[P][3] = grad_phi * d phi / d pose;
 * grad_edges[E][4] = sum over poses of grad_phi * d phi / d (stored A, B) rows.
 * grad_edges is overwritten.  Accumulation runs in pose order (deterministic).
 */
int oracle_psdf_backward(const double *footprint, int m, const double *edges, const int *offsets,
                         int M, const double *poses, long P, const oracle_params *prm,
                         const double *grad_phi, double *grad_pose, double *grad_edges,
                         int nthreads)
{
  int rc = check_inputs(m, offsets, M);
  if (rc) return rc;
  Ctx C;
  ctx_init(&C, footprint, m, edges, offsets, M, prm);
  int mx = max_obstacle_edges(offsets, M);
  long E = M > 0 ? offsets[M] : 0;
  if (grad_edges) memset(grad_edges, 0, sizeof(double) * 4 * (size_t)E);
  int *obs = (int *)malloc(sizeof(int) * (size_t)(P > 0 ? P : 1));
  double *ge = (double *)malloc(sizeof(double) * 4 * (size_t)mx * (size_t)(P > 0 ? P : 1));
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads)
#endif
  for (long q = 0; q < P; ++q) {
    PoseOut o;
    double *gq = ge + 4 * (size_t)mx * q;
    memset(gq, 0, sizeof(double) * 4 * (size_t)mx);
    eval_pose(&C, poses + 3 * q, &o, gq);
    obs[q] = o.obstacle;
    if (grad_pose) {
      grad_pose[3 * q] = grad_phi[q] * o.g[0];
      grad_pose[3 * q + 1] = grad_phi[q] * o.g[1];
      grad_pose[3 * q + 2] = grad_phi[q] * o.g[2];
    }
  }
  if (grad_edges) {
    for (long q = 0; q < P; ++q) {
      int i = obs[q];
      if (i < 0) continue;
      int e0 = offsets[i], n = offsets[i + 1] - e0;
      const double *gq = ge + 4 * (size_t)mx * q;
      for (int j = 0; j < n; ++j)
        for (int c = 0; c < 4; ++c) grad_edges[4 * (size_t)(e0 + j) + c] += grad_phi[q] * gq[4 * j + c];
    }
  }
  free(obs);
  free(ge);
  (void)nthreads;
  return 0;
}

/* Per-obstacle signed distances sd[P][M] (Sec. IV-D, before the min over
   obstacles); used to check the reduction and the tile bound. */
int oracle_psdf_obstacle_sd(const double *footprint, int m, const double *edges,
                            const int *offsets, int M, const double *poses, long P,
                            const oracle_params *prm, double *sd, int nthreads)
{
  int rc = check_inputs(m, offsets, M);
  if (rc) return rc;
  Ctx C;
  ctx_init(&C, footprint, m, edges, offsets, M, prm);
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads)
#endif
  for (long q = 0; q < P; ++q)
    for (int i = 0; i < M; ++i) {
      ObsOut ob;
      eval_obstacle(&C, i, poses + 3 * q, 0, &ob, NULL);
      sd[(size_t)q * M + i] = ob.sd;
    }
  (void)nthreads;
  return 0;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
