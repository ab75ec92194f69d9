// Scene preparation: Alg. 1 "EncodeEdges + upload" (Sec. IV-A.2), re-laid out
// for the B300 kernels.  Host code: validation (Assumption 1), sort-tile-
// recursive packing of obstacles into tiles, per-edge constants, upload.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "psdf_internal.h"

namespace psdf {

namespace {

uint32_t spread_bits(uint32_t x)
{
  x &= 0xffffu;
  x = (x | (x << 8)) & 0x00FF00FFu;
  x = (x | (x << 4)) & 0x0F0F0F0Fu;
  x = (x | (x << 2)) & 0x33333333u;
  x = (x | (x << 1)) & 0x55555555u;
  return x;
}

uint32_t morton2(uint32_t x, uint32_t y) { return spread_bits(x) | (spread_bits(y) << 1); }

// Check one obstacle against Assumption 1 and the layout rules.
int validate_obstacle(const float *rows, const ObsIn &o, int64_t idx)
{
  const float *e = rows + 4 * o.first_row;
  for (int k = 0; k < o.n; ++k)
    for (int c = 0; c < 4; ++c)
      if (!std::isfinite(e[4 * k + c]))
        return fail(PSDF_ERR_ARG, "obstacle " + std::to_string(idx) + ": non-finite coordinate");
  if (o.n == 2 || o.n < 1)
    return fail(PSDF_ERR_LAYOUT, "obstacle " + std::to_string(idx) +
                                     " has " + std::to_string(o.n) +
                                     " edges (1 = segment, >= 3 = closed polygon)");
  if (o.n > kMaxObsEdges)
    return fail(PSDF_ERR_CAPACITY, "obstacle " + std::to_string(idx) + " has more than " +
                                       std::to_string(kMaxObsEdges) + " edges");
  for (int k = 0; k < o.n; ++k) {
    double ux = (double)e[4 * k + 2] - e[4 * k], uy = (double)e[4 * k + 3] - e[4 * k + 1];
    if (std::sqrt(ux * ux + uy * uy) < 1e-6)
      return fail(PSDF_ERR_DEGENERATE_EDGE,
                  "edge row " + std::to_string(o.first_row + k) + " is shorter than 1e-6 m");
  }
  if (o.n >= 3) {
    double turn = 0.0;
    for (int k = 0; k < o.n; ++k) {
      int kn = (k + 1) % o.n;
      if (e[4 * k + 2] != e[4 * kn] || e[4 * k + 3] != e[4 * kn + 1])
        return fail(PSDF_ERR_LAYOUT, "obstacle " + std::to_string(idx) + ": B of edge row " +
                                         std::to_string(o.first_row + k) +
                                         " differs from A of the next edge (not closed)");
      double ux = (double)e[4 * k + 2] - e[4 * k], uy = (double)e[4 * k + 3] - e[4 * k + 1];
      double vx = (double)e[4 * kn + 2] - e[4 * kn], vy = (double)e[4 * kn + 3] - e[4 * kn + 1];
      double cr = ux * vy - uy * vx, dt = ux * vx + uy * vy;
      if (cr < 0.0)
        return fail(PSDF_ERR_LAYOUT, "obstacle " + std::to_string(idx) +
                                         " is not convex counter-clockwise");
      turn += std::atan2(cr, dt);
    }
    if (std::fabs(turn - 2.0 * M_PI) > 1e-6)
      return fail(PSDF_ERR_LAYOUT, "obstacle " + std::to_string(idx) +
                                       " does not turn exactly once (not a simple convex CCW polygon)");
  }
  return PSDF_OK;
}

}  // namespace

void free_scene(psdf_scene *s)
{
  if (!s) return;
  cudaFree(s->d_tiles);
  cudaFree(s->d_blob);
  cudaFree(s->d_vtx);
  cudaFree(s->d_far);
  cudaFree(s->d_row_obs);
  cudaFree(s->d_cell_off);
  cudaFree(s->d_cell_tiles);
  cudaFree(s->d_cell_aabbs);
  cudaFree(s->d_cell_info);
  cudaFree(s->d_cell_fab);
  cudaFree(s->d_cell_finfo);
  cudaFree(s->d_cull_obs);
  cudaFree(s->d_cand_circ);
  cudaFree(s->d_cand_rec);
  cudaFree(s->d_cand_rc);
  cudaFree(s->d_tile_ab);
  cudaFree(s->d_tile_info);
  delete s;
}

// rows: caller's edge rows [rows_total][4]; obstacles in caller order.
int build_host_scene(const float *rows, int64_t rows_total, const std::vector<ObsIn> &obs,
                     int tile_edges, const psdf_params *prm, HostScene *hs)
{
  const bool morton = (tile_edges & PSDF_TILE_MORTON) != 0;
  tile_edges &= ~PSDF_TILE_MORTON;
  if (tile_edges == 0) tile_edges = kDefaultTileEdges;
  if (tile_edges < 1 || tile_edges > kMaxTileEdges)
    return fail(PSDF_ERR_ARG, "tile_edges must be in [1, " + std::to_string(kMaxTileEdges) + "]");
  const double eps_seg = prm ? prm->eps_seg : 0.0;
  const double eps_axis = prm ? prm->eps_axis : 0.0;
  if (!(eps_seg >= 0.0) || !(eps_axis >= 0.0))
    return fail(PSDF_ERR_ARG, "eps_seg and eps_axis must be >= 0");
  const int M = (int)obs.size();
  int64_t n_edges = 0;
  int max_n = 0;
  for (int i = 0; i < M; ++i) {
    int rc = validate_obstacle(rows, obs[i], i);
    if (rc) return rc;
    n_edges += obs[i].n;
    max_n = std::max(max_n, obs[i].n);
    if (obs[i].first_row + obs[i].n - 1 > (int64_t)kMaxEdgeIndex)
      return fail(PSDF_ERR_CAPACITY, "edge rows above 2^24 - 1 do not fit the pair id");
  }
  if (max_n > tile_edges)
    return fail(PSDF_ERR_ARG, "an obstacle has more edges than tile_edges");

  // bounding box and obstacle centroids
  float bb[4] = {INFINITY, INFINITY, -INFINITY, -INFINITY};
  std::vector<double> cx(M), cy(M);
  for (int i = 0; i < M; ++i) {
    const float *e = rows + 4 * obs[i].first_row;
    double sx = 0, sy = 0;
    for (int k = 0; k < obs[i].n; ++k) {
      for (int c = 0; c < 2; ++c) {
        float x = e[4 * k + 2 * c], y = e[4 * k + 2 * c + 1];
        bb[0] = std::min(bb[0], x); bb[1] = std::min(bb[1], y);
        bb[2] = std::max(bb[2], x); bb[3] = std::max(bb[3], y);
      }
      sx += e[4 * k] + e[4 * k + 2];
      sy += e[4 * k + 1] + e[4 * k + 3];
    }
    cx[i] = sx / (2.0 * obs[i].n);
    cy[i] = sy / (2.0 * obs[i].n);
  }
  std::vector<int> order(M);
  std::iota(order.begin(), order.end(), 0);
  std::vector<int> tile_first;  // first sorted obstacle of each tile
  if (morton) {
    // greedy packing along a Morton (Z-order) curve of the centroids
    std::vector<uint32_t> code(M);
    double span = std::max((double)bb[2] - bb[0], (double)bb[3] - bb[1]);
    if (!(span > 0)) span = 1.0;
    for (int i = 0; i < M; ++i) {
      uint32_t qx = (uint32_t)std::min(65535.0, std::max(0.0, (cx[i] - bb[0]) / span * 65535.0));
      uint32_t qy = (uint32_t)std::min(65535.0, std::max(0.0, (cy[i] - bb[1]) / span * 65535.0));
      code[i] = morton2(qx, qy);
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return code[a] < code[b]; });
    int acc = 0;
    for (int s = 0; s < M; ++s) {
      const int n = obs[order[s]].n;
      if (s == 0 || acc + n > tile_edges) {
        tile_first.push_back(s);
        acc = 0;
      }
      acc += n;
    }
  } else {
    // Sort-tile-recursive packing: vertical slices of about equal edge count
    // along x, each slice ordered along y and cut greedily into tiles of at
    // most tile_edges edges.  Tiles come out close to square, which keeps their
    // AABBs (and the cull's lower bounds) tight.
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cx[a] < cx[b]; });
    const long long t_target = std::max<long long>(1, (n_edges + tile_edges - 1) / tile_edges);
    const int slices = std::max(1, (int)std::lround(std::sqrt((double)t_target)));
    const double per_slice = (double)n_edges / slices;
    {
      int s0 = 0;
      long long acc_edges = 0;
      for (int sl = 0; sl < slices && s0 < M; ++sl) {
        int s1 = s0;
        const double limit = per_slice * (sl + 1);
        while (s1 < M && (acc_edges + obs[order[s1]].n <= limit || s1 == s0 || sl == slices - 1)) {
          acc_edges += obs[order[s1]].n;
          ++s1;
        }
        std::stable_sort(order.begin() + s0, order.begin() + s1,
                         [&](int a, int b) { return cy[a] < cy[b]; });
        int acc = 0;
        for (int s = s0; s < s1; ++s) {
          const int n = obs[order[s]].n;
          if (s == s0 || acc + n > tile_edges) {
            tile_first.push_back(s);
            acc = 0;
          }
          acc += n;
        }
        s0 = s1;
      }
    }
  }
  const int T = (int)tile_first.size();
  tile_first.push_back(M);

  std::vector<TileHdr> tiles(T);
  std::vector<float4> vtx(2 * (size_t)n_edges);
  std::vector<int> far(n_edges);
  std::vector<ObsRec> row_obs(std::max<int64_t>(rows_total, 0), ObsRec{0, 0, 0, -1});
  std::vector<unsigned char> blob;
  std::vector<CullObs> cull_obs(M);
  std::vector<float4> tile_ab(T);
  std::vector<int4> tile_info(T);
  int64_t vglob = 0;
  int max_blob = 0, max_blob_ext = 0;
  for (int t = 0; t < T; ++t) {
    int s0 = tile_first[t], s1 = tile_first[t + 1];
    int nv = 0;
    for (int s = s0; s < s1; ++s) nv += obs[order[s]].n;
    const int nobs = s1 - s0;
    const int bytes = 16 * nobs + 32 * nv;
    TileHdr h;
    h.blob_off = (int)blob.size();
    h.blob_bytes = bytes;
    h.n_obs = nobs;
    h.n_vtx = nv;
    float ab[4] = {INFINITY, INFINITY, -INFINITY, -INFINITY};
    // the blob, then one bounding circle per obstacle (read by the cull only)
    blob.resize(blob.size() + bytes + 16 * nobs);
    float4 *circ = (float4 *)(blob.data() + h.blob_off + bytes);
    int4 *ob = (int4 *)(blob.data() + h.blob_off);
    float4 *vb = (float4 *)(blob.data() + h.blob_off + 16 * nobs);
    int vloc = 0;
    for (int s = s0; s < s1; ++s) {
      const ObsIn &o = obs[order[s]];
      const float *e = rows + 4 * o.first_row;
      ob[s - s0] = make_int4(vloc, o.n, (int)o.first_row, s);
      for (int k = 0; k < o.n; ++k)
        row_obs[o.first_row + k] = ObsRec{(int)vglob, o.n, (int)o.first_row, t};
      // obstacle vertex set: A of every edge, plus B for a segment
      const int nw = (o.n == 1) ? 2 : o.n;
      {
        // bounding circle: centre = vertex mean rounded to float, radius =
        // farthest vertex from that centre (FP64), rounded up
        double sx = 0.0, sy = 0.0;
        for (int q = 0; q < nw; ++q) {
          sx += (o.n == 1 && q == 1) ? (double)e[2] : (double)e[4 * q];
          sy += (o.n == 1 && q == 1) ? (double)e[3] : (double)e[4 * q + 1];
        }
        const float cxf = (float)(sx / nw), cyf = (float)(sy / nw);
        double r2 = 0.0;
        for (int q = 0; q < nw; ++q) {
          const double wx = ((o.n == 1 && q == 1) ? (double)e[2] : (double)e[4 * q]) - cxf;
          const double wy = ((o.n == 1 && q == 1) ? (double)e[3] : (double)e[4 * q + 1]) - cyf;
          r2 = std::max(r2, wx * wx + wy * wy);
        }
        const float rf = std::nextafter((float)std::sqrt(r2), INFINITY);
        // inner radius: the disc about the centre inside a closed polygon (its
        // distance to the nearest edge line), rounded down; 0 for a segment
        double rin = o.n >= 3 ? INFINITY : 0.0;
        for (int k = 0; k < o.n && o.n >= 3; ++k) {
          const double ax = e[4 * k], ay = e[4 * k + 1];
          const double ux = (double)e[4 * k + 2] - ax, uy = (double)e[4 * k + 3] - ay;
          const double dist = (ux * (cyf - ay) - uy * (cxf - ax)) / std::sqrt(ux * ux + uy * uy);
          rin = std::min(rin, dist);
        }
        const float rinf = rin > 1e-6 ? (float)(rin * (1.0 - 1e-5) - 1e-7) : 0.f;
        circ[s - s0] = make_float4(cxf, cyf, rf, rinf);
        cull_obs[s].circ = circ[s - s0];
        cull_obs[s].rec = make_int4((int)vglob, o.n, (int)o.first_row, t);
      }
      for (int k = 0; k < o.n; ++k) {
        double ax = e[4 * k], ay = e[4 * k + 1], bx = e[4 * k + 2], by = e[4 * k + 3];
        double ux = bx - ax, uy = by - ay;
        double len2 = ux * ux + uy * uy, len = std::sqrt(len2);
        double nxp = -uy / (len + eps_axis), nyp = ux / (len + eps_axis);
        double lo = INFINITY, hi = -INFINITY;
        int kfar = 0;
        for (int q = 0; q < nw; ++q) {
          double wx = (o.n == 1 && q == 1) ? (double)e[2] : (double)e[4 * q];
          double wy = (o.n == 1 && q == 1) ? (double)e[3] : (double)e[4 * q + 1];
          double pr = (wx - ax) * nxp + (wy - ay) * nyp;
          if (pr < lo) lo = pr;
          if (pr > hi) { hi = pr; kfar = q; }
        }
        if (o.n == 1) { lo = 0.0; hi = 0.0; kfar = 0; }
        float4 a = make_float4(e[4 * k], e[4 * k + 1], (float)(1.0 / (len2 + eps_seg)),
                               (float)(1.0 / (len + eps_axis)));
        float4 b = make_float4((float)lo, (float)hi, e[4 * k + 2], e[4 * k + 3]);
        vb[2 * (vloc + k)] = a;
        vb[2 * (vloc + k) + 1] = b;
        vtx[2 * (vglob + k)] = a;
        vtx[2 * (vglob + k) + 1] = b;
        far[vglob + k] = kfar;
        for (int c = 0; c < 2; ++c) {
          float x = e[4 * k + 2 * c], y = e[4 * k + 2 * c + 1];
          ab[0] = std::min(ab[0], x); ab[1] = std::min(ab[1], y);
          ab[2] = std::max(ab[2], x); ab[3] = std::max(ab[3], y);
        }
      }
      vloc += o.n;
      vglob += o.n;
    }
    std::memcpy(h.aabb, ab, sizeof(ab));
    tiles[t] = h;
    tile_ab[t] = make_float4(ab[0], ab[1], ab[2], ab[3]);
    tile_info[t] = make_int4(s0, nobs, nv, t);
    max_blob = std::max(max_blob, bytes);
    max_blob_ext = std::max(max_blob_ext, bytes + 16 * nobs);
  }

  hs->rows_total = rows_total;
  hs->M = M;
  hs->T = T;
  hs->tile_edges = tile_edges;
  hs->max_n = max_n;
  hs->n_edges = n_edges;
  std::memcpy(hs->bb, bb, sizeof(bb));
  if (M == 0) { hs->bb[0] = hs->bb[1] = hs->bb[2] = hs->bb[3] = 0.f; }
  hs->eps_seg = eps_seg;
  hs->eps_axis = eps_axis;
  hs->max_blob = max_blob;
  hs->max_blob_ext = max_blob_ext;
  hs->tiles.swap(tiles);
  hs->blob.swap(blob);
  hs->vtx.swap(vtx);
  hs->far.swap(far);
  hs->row_obs.swap(row_obs);
  hs->cull_obs.swap(cull_obs);
  hs->tile_ab.swap(tile_ab);
  hs->tile_info.swap(tile_info);
  return PSDF_OK;
}

// The cull's uniform grid (see CullGrid): cells about the size of a tile,
// reach one cell.  Host arithmetic in FP64; every tile is listed in each cell
// its AABB, widened by reach plus a margin, overlaps.  The margin covers the
// device's FP32 rounding of a pose's cell (relative error of a few 1e-7 of
// the coordinates' magnitude, plus that of 1/cs); reach_q takes it off twice.
// No grid when the lists would grow far beyond the tile count (strongly
// uneven tiles): lookups then scan all tiles.
void build_cull_grid(const HostScene &hs, CullGrid *g, float *cell, std::vector<int> *off,
                     std::vector<int> *tl, std::vector<float4> *ab, std::vector<int4> *info)
{
  *g = CullGrid();
  *cell = 0.f;
  off->clear();
  tl->clear();
  ab->clear();
  info->clear();
  const int T = hs.T;
  if (T == 0) return;
  const double x0 = hs.bb[0], y0 = hs.bb[1];
  const double W = (double)hs.bb[2] - x0, H = (double)hs.bb[3] - y0;
  double cs = std::sqrt(W * H / T);
  cs = std::max({cs, std::max(W, H) / 1000.0, 1e-3});
  const int nx = (int)std::floor(W / cs) + 1, ny = (int)std::floor(H / cs) + 1;
  const double reach = cs;
  const double mag = std::fabs(x0) + std::fabs(y0) + (nx + ny) * cs;
  const double margin = 1e-3 * cs + 1e-6 * mag;
  auto span = [&](double lo, double hi, int n, int *i0, int *i1) {
    *i0 = std::max(0, (int)std::floor((lo - reach - margin) / cs));
    *i1 = std::min(n - 1, (int)std::floor((hi + reach + margin) / cs));
  };
  std::vector<int> cnt((size_t)nx * ny + 1, 0);
  long long total = 0;
  for (int t = 0; t < T; ++t) {
    const float *a = hs.tiles[t].aabb;
    int i0, i1, j0, j1;
    span(a[0] - x0, a[2] - x0, nx, &i0, &i1);
    span(a[1] - y0, a[3] - y0, ny, &j0, &j1);
    for (int j = j0; j <= j1; ++j)
      for (int i = i0; i <= i1; ++i) ++cnt[(size_t)j * nx + i];
    total += (long long)std::max(0, i1 - i0 + 1) * std::max(0, j1 - j0 + 1);
  }
  if (total > 64LL * T + 65536) return;
  off->assign((size_t)nx * ny + 1, 0);
  for (size_t c = 0; c < (size_t)nx * ny; ++c) (*off)[c + 1] = (*off)[c] + cnt[c];
  tl->assign((size_t)total, 0);
  ab->assign((size_t)total, make_float4(0.f, 0.f, 0.f, 0.f));
  info->assign((size_t)total, make_int4(0, 0, 0, 0));
  std::vector<int> cur(off->begin(), off->end() - 1);
  for (int t = 0; t < T; ++t) {  // increasing t: every list sorted
    const float *a = hs.tiles[t].aabb;
    int i0, i1, j0, j1;
    span(a[0] - x0, a[2] - x0, nx, &i0, &i1);
    span(a[1] - y0, a[3] - y0, ny, &j0, &j1);
    for (int j = j0; j <= j1; ++j)
      for (int i = i0; i <= i1; ++i) {
        const int e = cur[(size_t)j * nx + i]++;
        (*tl)[e] = t;
        (*ab)[e] = make_float4(a[0], a[1], a[2], a[3]);
        (*info)[e] = hs.tile_info[t];
      }
  }
  g->x0 = hs.bb[0];
  g->y0 = hs.bb[1];
  g->inv_cs = (float)(1.0 / cs);
  g->reach_q = (float)(reach - 2.0 * margin);
  g->nx = nx;
  g->ny = ny;
  *cell = (float)cs;
}

// The candidate grid over the scene's bounding box: cells of side
// sqrt(kCand W H / (8 M)) (about kCand / 8 circle centres a cell), at most
// 2048 a side and 2^17 cells.  For every cell, the kCand obstacles of
// smallest near distance (to the cell widened by a margin for the rounding
// of a pose's FP32 cell index) and the radius rc below which no unlisted
// obstacle's near distance falls.  Obstacles whose circle is no larger than
// a cell are bucketed by their centre's cell and searched ring by ring (a
// centre r rings away lies at least (r - 1) cs from the cell, so its near
// distance is at least (r - 2) cs less the margins), up to kRingMax rings;
// larger ones are checked by every cell.  rc is the smaller of the
// (kCand + 1)-th near distance seen and that bound for the rings not
// searched, rounded down to FP32.
void build_cand_grid(const HostScene &hs, CandGrid *g, std::vector<float4> *circ,
                     std::vector<int4> *rec, std::vector<float> *rcv)
{
  *g = CandGrid();
  circ->clear();
  rec->clear();
  rcv->clear();
  const int M = (int)hs.cull_obs.size();
  if (M == 0) return;
  const double x0 = hs.bb[0], y0 = hs.bb[1];
  const double W = (double)hs.bb[2] - x0, H = (double)hs.bb[3] - y0;
  double cs = std::sqrt(kCand * std::max(W * H, 1e-12) / (8.0 * M));
  cs = std::max({cs, std::max(W, H) / 2047.0, 1e-3});
  while ((std::floor(W / cs) + 1) * (std::floor(H / cs) + 1) > (double)(1 << 17)) cs *= 1.25;
  const int nx = (int)std::floor(W / cs) + 1, ny = (int)std::floor(H / cs) + 1;
  const size_t cells = (size_t)nx * ny;
  const double mag = std::fabs(x0) + std::fabs(y0) + (nx + ny) * cs;
  const double margin = 1e-3 * cs + 1e-6 * mag;
  // small obstacles bucketed by the cell of their circle's centre
  std::vector<int> off(cells + 1, 0), ids, large;
  auto cell_of = [&](const float4 &cc) {
    const int i = std::min(nx - 1, std::max(0, (int)std::floor((cc.x - x0) / cs)));
    const int j = std::min(ny - 1, std::max(0, (int)std::floor((cc.y - y0) / cs)));
    return (size_t)j * nx + i;
  };
  for (int o = 0; o < M; ++o) {
    const float4 cc = hs.cull_obs[o].circ;
    if (cc.z > cs) large.push_back(o);
    else ++off[cell_of(cc) + 1];
  }
  if ((double)large.size() * (double)cells > 2e8) return;  // no grid: the tile path serves
  for (size_t c = 0; c < cells; ++c) off[c + 1] += off[c];
  ids.resize(off[cells]);
  {
    std::vector<int> cur(off.begin(), off.end() - 1);
    for (int o = 0; o < M; ++o) {
      const float4 cc = hs.cull_obs[o].circ;
      if (!(cc.z > cs)) ids[cur[cell_of(cc)]++] = o;
    }
  }
  constexpr int K1 = kCand + 1;
  constexpr int kRingMax = 16;
  circ->assign(cells * kCand, make_float4(0.f, 0.f, INFINITY, -INFINITY));
  rec->assign(cells * kCand, make_int4(0, 0, 0, -1));
  rcv->assign(cells, INFINITY);
  for (int cj = 0; cj < ny; ++cj)
    for (int ci = 0; ci < nx; ++ci) {
      const double bx0 = x0 + ci * cs - margin, bx1 = x0 + (ci + 1) * cs + margin;
      const double by0 = y0 + cj * cs - margin, by1 = y0 + (cj + 1) * cs + margin;
      double bd[K1];
      int bo[K1], nb = 0;
      auto offer = [&](int o) {
        const float4 cc = hs.cull_obs[o].circ;
        const double dx = std::max({bx0 - cc.x, (double)cc.x - bx1, 0.0});
        const double dy = std::max({by0 - cc.y, (double)cc.y - by1, 0.0});
        const double nd = std::sqrt(dx * dx + dy * dy) - cc.z;
        if (nb == K1 && !(nd < bd[K1 - 1])) return;
        int k = nb < K1 ? nb++ : K1 - 1;
        while (k > 0 && bd[k - 1] > nd) {
          bd[k] = bd[k - 1];
          bo[k] = bo[k - 1];
          --k;
        }
        bd[k] = nd;
        bo[k] = o;
      };
      for (int o : large) offer(o);
      double unseen = INFINITY;  // bound on the near distance of every obstacle not offered
      for (int r = 0;; ++r) {
        const double lb_r = (r - 2) * cs - 2 * margin;  // every small obstacle r or more rings away
        if (nb == K1 && lb_r > bd[K1 - 1]) break;
        if (r > std::max(nx, ny)) break;  // every cell searched
        if (r > kRingMax) {
          unseen = lb_r;
          break;
        }
        for (int j = cj - r; j <= cj + r; ++j) {
          if (j < 0 || j >= ny) continue;
          const bool full_row = (r == 0 || j == cj - r || j == cj + r);
          for (int i = ci - r; i <= ci + r; i += full_row ? 1 : 2 * r) {
            if (i < 0 || i >= nx) continue;
            const size_t c = (size_t)j * nx + i;
            for (int e = off[c]; e < off[c + 1]; ++e) offer(ids[e]);
          }
        }
      }
      const size_t c = (size_t)cj * nx + ci;
      for (int k = 0; k < std::min(nb, kCand); ++k) {
        (*circ)[c * kCand + k] = hs.cull_obs[bo[k]].circ;
        (*rec)[c * kCand + k] = hs.cull_obs[bo[k]].rec;
      }
      double rc = std::min(nb == K1 ? bd[K1 - 1] : INFINITY, unseen);
      float rf = (float)rc;
      if ((double)rf > rc) rf = std::nextafter(rf, -INFINITY);
      (*rcv)[c] = rf;
    }
  g->x0 = hs.bb[0];
  g->y0 = hs.bb[1];
  g->inv_cs = (float)(1.0 / cs);
  g->nx = nx;
  g->ny = ny;
}

int build_scene(const float *rows, int64_t rows_total, const std::vector<ObsIn> &obs,
                int tile_edges, const psdf_params *prm, cudaStream_t st, psdf_scene **out)
{
  HostScene hs;
  int rc = build_host_scene(rows, rows_total, obs, tile_edges, prm, &hs);
  if (rc) return rc;
  psdf_scene *s = new psdf_scene();
  s->rows_total = hs.rows_total;
  s->M = hs.M;
  s->n_tiles = hs.T;
  s->tile_edges = hs.tile_edges;
  s->max_obs_edges = hs.max_n;
  s->n_edges = hs.n_edges;
  std::memcpy(s->bbox, hs.bb, sizeof(hs.bb));
  s->eps_seg = (float)hs.eps_seg;
  s->eps_axis = (float)hs.eps_axis;
  s->max_blob_bytes = hs.max_blob;
  s->max_blob_ext_bytes = hs.max_blob_ext;
  cudaGetDevice(&s->device);
  if (!rc) rc = dev_upload(&s->d_tiles, hs.tiles, st, &s->device_bytes);
  if (!rc) rc = dev_upload(&s->d_blob, hs.blob, st, &s->device_bytes);
  if (!rc) rc = dev_upload(&s->d_vtx, hs.vtx, st, &s->device_bytes);
  if (!rc) rc = dev_upload(&s->d_far, hs.far, st, &s->device_bytes);
  if (!rc) rc = dev_upload(&s->d_row_obs, hs.row_obs, st, &s->device_bytes);
  if (!rc) rc = dev_upload(&s->d_cull_obs, hs.cull_obs, st, &s->device_bytes);
  if (!rc) rc = dev_upload(&s->d_tile_ab, hs.tile_ab, st, &s->device_bytes);
  if (!rc) rc = dev_upload(&s->d_tile_info, hs.tile_info, st, &s->device_bytes);
  {
    std::vector<float4> cand_circ;
    std::vector<int4> cand_rec;
    std::vector<float> cand_rc;
    build_cand_grid(hs, &s->cand, &cand_circ, &cand_rec, &cand_rc);
    if (!rc && s->cand.nx > 0) {
      rc = dev_upload(&s->d_cand_circ, cand_circ, st, &s->device_bytes);
      if (!rc) rc = dev_upload(&s->d_cand_rec, cand_rec, st, &s->device_bytes);
      if (!rc) rc = dev_upload(&s->d_cand_rc, cand_rc, st, &s->device_bytes);
      s->cand.circ = s->d_cand_circ;
      s->cand.rec = s->d_cand_rec;
      s->cand.rc = s->d_cand_rc;
    }
  }
  std::vector<int> cell_off, cell_tiles;
  std::vector<float4> cell_aabbs;
  std::vector<int4> cell_info;
  build_cull_grid(hs, &s->grid, &s->grid_cell, &cell_off, &cell_tiles, &cell_aabbs, &cell_info);
  s->grid_entries = (int64_t)cell_tiles.size();
  if (!rc && s->grid.nx > 0) {
    rc = dev_upload(&s->d_cell_off, cell_off, st, &s->device_bytes);
    if (!rc) rc = dev_upload(&s->d_cell_tiles, cell_tiles, st, &s->device_bytes);
    if (!rc) rc = dev_upload(&s->d_cell_aabbs, cell_aabbs, st, &s->device_bytes);
    if (!rc) rc = dev_upload(&s->d_cell_info, cell_info, st, &s->device_bytes);
    s->grid.off = s->d_cell_off;
    s->grid.tl = s->d_cell_tiles;
    s->grid.ab = s->d_cell_aabbs;
    s->grid.info = s->d_cell_info;
    // fixed-capacity copies when every list is short (a multiple of 16 slots)
    int longest = 0;
    for (size_t c = 0; c + 1 < cell_off.size(); ++c)
      longest = std::max(longest, cell_off[c + 1] - cell_off[c]);
    const int cap = (longest + 15) / 16 * 16;
    if (!rc && cap > 0 && cap <= 64) {
      const size_t cells = cell_off.size() - 1;
      std::vector<float4> fab(cells * cap, make_float4(INFINITY, INFINITY, -INFINITY, -INFINITY));
      std::vector<int4> finfo(cells * cap, make_int4(0, 0, 0, -2));
      for (size_t c = 0; c < cells; ++c)
        for (int e = cell_off[c]; e < cell_off[c + 1]; ++e) {
          fab[c * cap + (e - cell_off[c])] = cell_aabbs[e];
          finfo[c * cap + (e - cell_off[c])] = cell_info[e];
        }
      rc = dev_upload(&s->d_cell_fab, fab, st, &s->device_bytes);
      if (!rc) rc = dev_upload(&s->d_cell_finfo, finfo, st, &s->device_bytes);
      if (!rc) {
        s->grid.cap = cap;
        s->grid.fab = s->d_cell_fab;
        s->grid.finfo = s->d_cell_finfo;
      }
    }
  }
  if (!rc) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_fail(e, "scene upload");
  }
  if (rc) {
    free_scene(s);
    return rc;
  }
  *out = s;
  return PSDF_OK;
}

}  // namespace psdf

using namespace psdf;

extern "C" int psdf_scene_create_csr(const float *edges, const int32_t *offsets, int32_t M,
                                     int32_t tile_edges, const psdf_params *params,
                                     void *stream, psdf_scene **out)
{
  if (!out) return fail(PSDF_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (M < 0) return fail(PSDF_ERR_ARG, "M < 0");
  if (!offsets) return fail(PSDF_ERR_ARG, "offsets is NULL");
  if (offsets[0] != 0) return fail(PSDF_ERR_LAYOUT, "offsets[0] must be 0");
  std::vector<ObsIn> obs(M);
  for (int i = 0; i < M; ++i) {
    if (offsets[i + 1] < offsets[i]) return fail(PSDF_ERR_LAYOUT, "offsets decrease");
    obs[i] = ObsIn{offsets[i], offsets[i + 1] - offsets[i]};
  }
  int64_t E = offsets[M];
  if (E > 0 && !edges) return fail(PSDF_ERR_ARG, "edges is NULL");
  return build_scene(edges, E, obs, tile_edges, params, (cudaStream_t)stream, out);
}

extern "C" int psdf_scene_create_padded(const float *A, const float *B, const uint8_t *S,
                                        int32_t Mbar, int32_t mbar, int32_t tile_edges,
                                        const psdf_params *params, void *stream,
                                        psdf_scene **out)
{
  if (!out) return fail(PSDF_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (Mbar < 0 || mbar < 0) return fail(PSDF_ERR_ARG, "negative padded size");
  int64_t rows_total = (int64_t)Mbar * mbar;
  if (rows_total > 0 && (!A || !B || !S)) return fail(PSDF_ERR_ARG, "A, B or S is NULL");
  std::vector<float> rows(4 * (size_t)rows_total);
  std::vector<ObsIn> obs;
  for (int i = 0; i < Mbar; ++i) {
    int n = 0;
    bool gap = false;
    for (int j = 0; j < mbar; ++j) {
      int64_t r = (int64_t)i * mbar + j;
      rows[4 * r] = A[2 * r];
      rows[4 * r + 1] = A[2 * r + 1];
      rows[4 * r + 2] = B[2 * r];
      rows[4 * r + 3] = B[2 * r + 1];
      if (S[r] > 1) return fail(PSDF_ERR_LAYOUT, "mask S holds a value other than 0 or 1");
      if (S[r]) {
        if (gap) return fail(PSDF_ERR_LAYOUT, "valid mask entries of a row must come first");
        ++n;
      } else {
        gap = true;
      }
    }
    if (n > 0) obs.push_back(ObsIn{(int64_t)i * mbar, n});
  }
  return build_scene(rows.data(), rows_total, obs, tile_edges, params, (cudaStream_t)stream, out);
}

extern "C" int psdf_scene_destroy(psdf_scene *scene)
{
  free_scene(scene);
  return PSDF_OK;
}

extern "C" int psdf_scene_cull_grid(const psdf_scene *s, psdf_cull_grid_info *info)
{
  if (!s || !info) return fail(PSDF_ERR_ARG, "scene or info is NULL");
  info->nx = s->grid.nx;
  info->ny = s->grid.ny;
  info->entries = s->grid.nx > 0 ? s->grid_entries : 0;
  info->x0 = s->grid.x0;
  info->y0 = s->grid.y0;
  info->cell = s->grid.nx > 0 ? s->grid_cell : 0.f;
  info->reach = s->grid.nx > 0 ? s->grid.reach_q : 0.f;
  info->inv_cell = s->grid.inv_cs;
  return PSDF_OK;
}

extern "C" int psdf_scene_cull_grid_copy(const psdf_scene *s, int32_t *offsets, int32_t *tiles,
                                         float *aabbs)
{
  if (!s) return fail(PSDF_ERR_ARG, "scene is NULL");
  cudaError_t e = cudaSuccess;
  if (s->grid.nx > 0) {
    if (!offsets || !tiles) return fail(PSDF_ERR_ARG, "offsets or tiles is NULL");
    const size_t cells = (size_t)s->grid.nx * s->grid.ny + 1;
    e = cudaMemcpy(offsets, s->d_cell_off, 4 * cells, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && s->grid_entries > 0)
      e = cudaMemcpy(tiles, s->d_cell_tiles, 4 * (size_t)s->grid_entries, cudaMemcpyDeviceToHost);
  }
  if (e == cudaSuccess && aabbs && s->n_tiles > 0) {
    std::vector<TileHdr> h(s->n_tiles);
    e = cudaMemcpy(h.data(), s->d_tiles, sizeof(TileHdr) * h.size(), cudaMemcpyDeviceToHost);
    for (size_t t = 0; e == cudaSuccess && t < h.size(); ++t)
      std::memcpy(aabbs + 4 * t, h[t].aabb, sizeof(h[t].aabb));
  }
  return e == cudaSuccess ? PSDF_OK : cuda_fail(e, "cudaMemcpy(cull grid)");
}

extern "C" int psdf_scene_get_info(const psdf_scene *s, psdf_scene_info *info)
{
  if (!s || !info) return fail(PSDF_ERR_ARG, "scene or info is NULL");
  info->n_edges = s->n_edges;
  info->n_obstacles = s->M;
  info->n_tiles = s->n_tiles;
  info->tile_edges = s->tile_edges;
  info->max_obstacle_edges = s->max_obs_edges;
  std::memcpy(info->bbox, s->bbox, sizeof(s->bbox));
  info->device_bytes = (int64_t)s->device_bytes;
  return PSDF_OK;
}
