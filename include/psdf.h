/*
 * psdf.h -- C ABI of the B300 (sm_103a) Polygonal Signed Distance Function
 * library, libpsdf_b300.so.
 *
 * The library evaluates the PSDF of "GPU-Accelerated Polygonal Signed
 * Distance Functions for Real-Time Collision Avoidance": the signed distance
 * phi(x, E) between a convex polygonal robot footprint posed at
 * x = (px, py, theta) and a set of obstacle boundary edges E, plus its
 * gradient (Sec. III-B, Sec. IV, Alg. 1 PSDF_Forward / PSDF_Backward).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - All floating point data is IEEE float32; all arithmetic on the device is
 *    float32.
 *  - Footprint: HOST pointer, float[m][2], the robot polygon in its local
 *    frame, counter-clockwise, strictly convex, 3 <= m <= 16 (Assumption 1,
 *    Sec. IV-A.1).  The library copies it by value into every launch.
 *  - Poses and all per-pose outputs are DEVICE pointers owned by the caller:
 *    poses float[P][3] = (px, py, theta); phi float[P]; dphi float[P][3];
 *    active uint32[P].  The library never allocates caller outputs.  Pinned
 *    host memory mapped into the device's address space at the same address
 *    (cudaHostAlloc / cudaMallocHost with unified addressing) is accepted as
 *    well: the kernels then read the poses and write the outputs across the
 *    host link themselves, with no copy call (zero-copy).  Any other host
 *    pointer for the poses is rejected (PSDF_ERR_ARG).
 *  - Every evaluation call is asynchronous on `stream` (a cudaStream_t passed
 *    as void*, NULL = the legacy default stream); nothing is read back to the
 *    host and no device memory is allocated, so calls can be captured in a
 *    CUDA graph after the scene exists.
 *  - Return value: PSDF_OK (0) or one of the PSDF_ERR_* codes below.  Nothing
 *    throws across the ABI; psdf_last_error() returns a message for the last
 *    failing call on the calling thread.  Argument errors are detected on the
 *    host before anything is launched.
 *
 * Active pair id (uint32): (edge << 8) | (kind << 4) | l, where `edge` is the
 * edge index in the caller's original numbering (CSR row, or i * mbar + j for
 * the padded layout), `l` a robot vertex / edge / axis index and `kind`:
 *   0 robot vertex l -> obstacle edge (closest point on [A, B), or B for a
 *     one-edge obstacle)               1 obstacle vertex A -> robot edge l
 *   2 one-edge obstacle's B -> robot edge l
 *   3/4 robot axis l: overlap = obstacle max - robot min / robot max -
 *     obstacle min, extreme obstacle vertex A of `edge`      5/6 same, B
 *   7/8 obstacle axis of `edge`: overlap = obstacle max - robot min (robot
 *     extreme vertex l) / robot max - obstacle min (robot extreme vertex l).
 * Among equal values the lowest (value, id) wins; across obstacles the one
 * whose first edge has the lowest original index.  0xFFFFFFFF = none (empty
 * scene).  Separated distances are compared through their squares.
 */
#ifndef PSDF_H
#define PSDF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define PSDF_OK 0
#define PSDF_ERR_ARG 1             /* null pointer, negative or oversize count  */
#define PSDF_ERR_FOOTPRINT 2       /* m outside [3,16], not CCW strictly convex */
#define PSDF_ERR_DEGENERATE_EDGE 3 /* an edge shorter than 1e-6 m               */
#define PSDF_ERR_LAYOUT 4          /* bad offsets / mask, unclosed or non-convex
                                      polygon, 2-edge obstacle                  */
#define PSDF_ERR_CUDA 5            /* a CUDA runtime call failed                */
#define PSDF_ERR_TIMEOUT 6         /* a bounded device-side wait ran out        */
#define PSDF_ERR_CAPACITY 7        /* workspace too small / size limit exceeded */

#define PSDF_PAIR_NONE 0xFFFFFFFFu
#define PSDF_MAX_FOOTPRINT 16
#define PSDF_MAX_OBSTACLE_EDGES 256
/* OR into tile_edges of psdf_scene_create_*: pack tiles greedily along a
 * Morton (Z-order) curve of the obstacle centroids instead of the default
 * sort-tile-recursive order (tiles then follow the curve and may be long) */
#define PSDF_TILE_MORTON 0x10000

typedef struct psdf_scene psdf_scene; /* opaque: owns the device copy of E  */

/* Tolerances of Sec. IV-B / IV-C.  eps_seg: epsilon added to |v|^2 in the
 * projection factor u; eps_axis: epsilon added to |u| in the obstacle-axis
 * normal; eps_sat: the separating-axis tolerance.  eta = 0 selects the hard
 * minimum of the overlaps (the exact penetration depth, Sec. IV-C); eta > 0
 * the log-sum-exp soft minimum of Eq. penetration_depth over all of an
 * obstacle's axes (psdf_eval, psdf_eval_grad, psdf_backward, the
 * no-allocation call, psdf_eval_culled and the batched plans; the tile
 * helpers take the hard minimum only and reject eta > 0).  With eta > 0 a non-separated
 * obstacle's sd = -pen_soft (which is positive for shallow overlaps), its
 * gradient is the softmax-weighted sum over its axes with delta > 0, and the
 * active pair id still names the hard minimum's pair.  eta must be finite
 * and >= 0 (PSDF_ERR_ARG otherwise). */
typedef struct {
  float eps_seg;
  float eps_axis;
  float eps_sat;
  float eta;
} psdf_params;

typedef struct {
  int64_t n_edges;
  int32_t n_obstacles;
  int32_t n_tiles;
  int32_t tile_edges;   /* maximum edges per tile                         */
  int32_t max_obstacle_edges;
  float bbox[4];        /* xmin, ymin, xmax, ymax of all endpoints          */
  int64_t device_bytes; /* device memory owned by the scene                 */
} psdf_scene_info;

/* Message for the last failing call on this thread ("" if none). */
const char *psdf_last_error(void);

/* ABI version (major * 100 + minor). */
int psdf_version(void);

/* ---- scene preparation (Alg. 1 EncodeEdges + upload, Sec. IV-A.2) -------
 * Validates the edge set, packs the obstacles into tiles of at most
 * `tile_edges` edges (0 selects 256; no obstacle straddles a tile) by
 * sort-tile-recursive order of their centroids (vertical slices along x,
 * each ordered along y), precomputes per-edge constants and uploads
 * everything to the current device (synchronously, on `stream`).
 *
 * psdf_scene_create_csr: edges HOST float[E][4] rows (Ax, Ay, Bx, By) in the
 * world frame; offsets HOST int32[M+1], obstacle i owns rows
 * offsets[i] .. offsets[i+1]-1 (offsets[0] = 0, non-decreasing).  An obstacle
 * is a single segment (1 edge) or a closed convex CCW polygon (>= 3 edges,
 * B of each edge bit-equal to A of the next, wrapping around).  M = 0 gives an
 * empty scene (phi = +inf).
 *
 * psdf_scene_create_padded: the paper's padded tensors A, B HOST
 * float[Mbar][mbar][2] and mask S HOST uint8[Mbar][mbar]; the valid entries of
 * each row must come first; rows with no valid entry are skipped.  Pair ids
 * report i * mbar + j.
 *
 * `params` (nullable = all zero) fixes eps_seg and eps_axis, which enter the
 * per-edge precompute (1 / (|u|^2 + eps_seg), 1 / (|u| + eps_axis)); every
 * evaluation of the scene must pass the same two values (else PSDF_ERR_ARG).
 * eps_sat and eta are free per call.
 *
 * The scene is freed with psdf_scene_destroy (NULL is accepted).  A scene may
 * be evaluated from several streams at once; it is never written after
 * creation. */
int psdf_scene_create_csr(const float *edges, const int32_t *offsets, int32_t M,
                          int32_t tile_edges, const psdf_params *params, void *stream,
                          psdf_scene **out);
int psdf_scene_create_padded(const float *A, const float *B, const uint8_t *S, int32_t Mbar,
                             int32_t mbar, int32_t tile_edges, const psdf_params *params,
                             void *stream, psdf_scene **out);
int psdf_scene_destroy(psdf_scene *scene);
int psdf_scene_get_info(const psdf_scene *scene, psdf_scene_info *info);

/* ---- workspace ----------------------------------------------------------
 * Device scratch needed by psdf_eval / psdf_eval_grad for P poses (one
 * 64-bit min-key per pose, plus an error word).  The caller allocates it
 * (>= 256-byte aligned) and may reuse it across calls on the same stream;
 * calls that overlap on the GPU need separate workspaces. */
size_t psdf_workspace_bytes(int64_t P);

/* Synchronizes `stream` and reports a device-side failure recorded in the
 * workspace by the last evaluation: PSDF_ERR_TIMEOUT if a bounded wait ran
 * out (the affected poses then hold phi = NaN, active = PSDF_PAIR_NONE),
 * else PSDF_OK. */
int psdf_workspace_status(const void *workspace, void *stream);

/* ---- PSDF_Forward (Alg. 1; Sec. IV-A.3 stages 1-4, Eq. psdf_value) -------
 * phi[p] = min over obstacles of sd(P0(x_p), P_i) for every pose.  `active`
 * (nullable) receives the active pair id.  Full scan over every edge tile. */
int psdf_eval(const float *footprint, int32_t m, const psdf_scene *scene, const float *poses,
              int64_t P, const psdf_params *params, float *phi, uint32_t *active,
              void *workspace, size_t workspace_bytes, void *stream);

/* Value and gradient d phi / d (px, py, theta) through the active pair
 * (the active-branch subgradient of Sec. IV-D; Alg. 1 PSDF_Backward with a
 * unit seed).  dphi is float[P][3]; active is nullable. */
int psdf_eval_grad(const float *footprint, int32_t m, const psdf_scene *scene,
                   const float *poses, int64_t P, const psdf_params *params, float *phi,
                   float *dphi, uint32_t *active, void *workspace, size_t workspace_bytes,
                   void *stream);

/* ---- scene parts: keys, their minimum, the owner's epilogue --------------
 * Eq. psdf_value is a minimum over obstacles, so a scene may be split into
 * parts whose caller rows are consecutive ranges of one numbering (part r a
 * CSR scene of its own holding the whole scene's rows row_offset_r ..
 * row_offset_r + rows_r - 1): a static map and each step's moving obstacles
 * (Sec. V, time-varying edge sets), or an edge set sharded over GPUs.  Each
 * part yields per-pose 64-bit keys (ordered value << 32 | rank, the rank
 * being the whole scene's row of the obstacle's first edge), their minimum
 * is the whole scene's key with its tie-break, and the part that holds the
 * winning obstacle runs the epilogue: the outputs equal one evaluation of
 * the whole scene bit for bit.
 *
 * psdf_eval_keys: keys[P] (DEVICE uint64, caller-owned, overwritten) of the
 *   part by the full scan, ranks offset by row_offset; 0xFFFF...F = no
 *   obstacle.  workspace: DEVICE, >= 256 bytes, 256-byte aligned (only its
 *   error word is used; psdf_workspace_status reads it).
 * psdf_merge_keys: b[p] = min(a[p], b[p]) for DEVICE uint64 a, b.  Across
 *   GPUs the same minimum is one all-reduce: the keys read as int64 with the
 *   top bit flipped order as the unsigned keys do.
 * psdf_finish_keys: the epilogue (phi, active pair in the whole scene's row
 *   numbering, gradient if dphi) of the poses whose merged key names an
 *   obstacle of this part, and, when own_empty != 0, of the poses whose key
 *   names none (phi = +inf, active = PSDF_PAIR_NONE); the other poses'
 *   outputs are not written.  dphi and active are nullable.
 * All are asynchronous on `stream` and allocate nothing.  row_offset >= 0
 * and row_offset + the part's rows must fit the pair id's 24-bit edge field
 * (PSDF_ERR_ARG otherwise). */
int psdf_eval_keys(const float *footprint, int32_t m, const psdf_scene *scene, const float *poses,
                   int64_t P, const psdf_params *params, int64_t row_offset, uint64_t *keys,
                   void *workspace, size_t workspace_bytes, void *stream);
int psdf_merge_keys(const uint64_t *a, uint64_t *b, int64_t P, void *stream);
int psdf_finish_keys(const float *footprint, int32_t m, const psdf_scene *scene,
                     const float *poses, int64_t P, const psdf_params *params,
                     int64_t row_offset, int32_t own_empty, const uint64_t *keys, float *phi,
                     float *dphi, uint32_t *active, void *stream);

/* ---- SQP-RTI stage parameters (Alg. 1, PSDF-MPC pipeline) ---------------
 * The affine safety constraint of every prediction stage, J_g dx <= h, from
 * the linearization of h = phi - d_min at the nominal pose (Sec. V-A):
 * stage float[P][4] = {h, J_g} with h = phi - d_min and J_g = -d phi / d x
 * (x = (px, py, theta)); active (optional) as for psdf_eval.  The same
 * kernels as psdf_eval_grad with the conversion fused into the per-pose
 * epilogue (phi and the gradient are not stored separately); d_min must be
 * finite.  Asynchronous, no allocation (graph-capturable). */
int psdf_stage_params(const float *footprint, int32_t m, const psdf_scene *scene,
                      const float *poses, int64_t P, const psdf_params *params, float d_min,
                      float *stage, uint32_t *active, void *workspace, size_t workspace_bytes,
                      void *stream);

/* ---- backward (vector-Jacobian product of phi, Sec. IV-D) ----------------
 * Given the active pair ids of a previous psdf_eval / psdf_eval_grad with the
 * same footprint, scene, poses and params, and an upstream gradient
 * grad_phi[P]:
 *   grad_pose[p][k] = grad_phi[p] * d phi_p / d pose_p[k]   (overwritten;
 *                                                             nullable)
 *   grad_edges[e][c] += sum_p grad_phi[p] * d phi_p / d edges[e][c]
 *                       (accumulated; nullable; float[E][4] in the caller's
 *                        original row order: CSR rows, or Mbar*mbar rows for a
 *                        padded scene)
 * A closed polygon's vertex is stored twice (A of its edge, B of the previous
 * edge); its gradient is reported in the A slot and the B slots of closed
 * polygons stay zero (the derivative with respect to one copy alone is not
 * defined).  A one-edge obstacle's A and B get their own gradients.
 * Accumulation into grad_edges uses float atomics (summation order varies). */
int psdf_backward(const float *footprint, int32_t m, const psdf_scene *scene,
                  const float *poses, int64_t P, const psdf_params *params,
                  const uint32_t *active, const float *grad_phi, float *grad_pose,
                  float *grad_edges, void *stream);

/* ---- backward from records saved by the forward (hard minimum) -----------
 * The forward's epilogue already takes the active pair's gradient (Alg. 1,
 * value + gradient); these calls keep, per pose, what the backward above
 * recomputes from the active pair id, so that the backward is a scale and a
 * scatter.  Record layout, float saved[P][16] (DEVICE, 16-byte aligned,
 * caller-owned, written by the forward, read by psdf_backward_saved):
 *   0..2  d phi / d (x, y, theta), the dphi the forward writes
 *   3     int32 bits: the count (0..3) of edge-endpoint rows below, or -1
 *         when the pose has no gradient (no obstacle, or touching without
 *         overlap on the active axis)
 *   4 + 3i, 5 + 3i, 6 + 3i (i < 3): int32 bits of (caller edge row * 4 +
 *         column), then d phi / d column, d phi / d (column + 1); column 0 is
 *         (Ax, Ay), column 2 is (Bx, By), as in grad_edges
 *   13..15 zero
 * psdf_eval_grad_save / psdf_eval_culled_save: psdf_eval_grad /
 * psdf_eval_culled plus the records (dphi and saved required); eta > 0 is
 * rejected (PSDF_ERR_ARG: the soft backward touches every axis of the
 * obstacle).  psdf_backward_saved: grad_pose and grad_edges exactly as
 * psdf_backward computes them from the same forward (grad_pose bit for bit;
 * grad_edges up to the order of its float atomics); rows outside the
 * scene's 4 * rows_total columns are skipped.  All three are asynchronous
 * on `stream` and allocate nothing (graph-capturable). */
int psdf_eval_grad_save(const float *footprint, int32_t m, const psdf_scene *scene,
                        const float *poses, int64_t P, const psdf_params *params, float *phi,
                        float *dphi, uint32_t *active, float *saved, void *workspace,
                        size_t workspace_bytes, void *stream);
int psdf_backward_saved(const psdf_scene *scene, const float *saved, int64_t P,
                        const float *grad_phi, float *grad_pose, float *grad_edges,
                        void *stream);

/* ---- exact tile cull with a proposal (learned or bound-ordered) or the
 * scene's candidate grid ---------------------------------------------------
 * Same outputs as psdf_eval_grad, bit for bit, while evaluating only part of
 * the (pose, obstacle) pairs (the exact value of Eq. psdf_value, Sec. IV-D,
 * over the obstacles that can attain it).  Each pose first takes an upper
 * bound UB >= phi from obstacle circles (a circle containing the obstacle,
 * and a disc inside it): under PSDF_PROPOSE_BOUND and PSDF_PROPOSE_MLP from
 * the circles of the obstacles of its k proposed tiles -- the k tiles of
 * smallest bound (BOUND), or the network's k tiles of smallest predicted
 * signed distance among the 8 of smallest bound (MLP), among the tiles of
 * the pose's cell in the scene's cull grid (every tile within one cell size
 * of the pose; all tiles for a pose outside the grid); under
 * PSDF_PROPOSE_CIRCLES from the 32 candidate obstacles the scene keeps for
 * the pose's cell of its candidate grid (the obstacles whose circles come
 * nearest the cell, chosen when the scene is built, and a completeness
 * radius: no unlisted obstacle's circle comes within it of the cell).  A pose in its
 * candidate cell whose UB plus the footprint radius lies within that radius
 * needs only the candidates.  Any other pose lists every tile whose
 * conservative lower bound
 *     LB = dist(p, tile AABB) - r_foot - (1e-4 + 1e-5 dist)
 * does not exceed UB ("fallback" pairs; all listed pairs are fallback pairs
 * under PSDF_PROPOSE_CIRCLES), taken from the cull grid cell's list when
 * those tiles all lie within its reach, else from all tiles.  The obstacles
 * whose circle bound exceeds UB are skipped, the rest are evaluated exactly.
 * No skipped tile or obstacle can hold a smaller value or a tie, so phi, the
 * active pair and the gradient equal the full scan's.  The proposal only
 * changes how much work the exact part does.  One launch: 16 poses a CTA (8
 * under PSDF_PROPOSE_CIRCLES), each pose's ranking and bound by 16 lanes,
 * the tile tests, circle tests and exact evaluations shared out over the
 * CTA.  phi, dphi and active may be pinned, device-mapped host memory; each
 * CTA writes them as contiguous blocks. */
typedef struct psdf_mlp psdf_mlp; /* opaque: tile-proposal network (device) */

/* The cull grid of a scene: a uniform grid of nx x ny square cells of side
 * `cell` metres from (x0, y0), built with the scene; each cell lists every
 * tile whose AABB comes within `cell` of it (`entries` list entries in all).
 * A pose uses its cell's list while the tiles it needs lie within `reach`
 * metres.  nx = ny = 0: no grid (a scene without tiles, or one whose tiles'
 * AABBs are so large that the lists would exceed 64 entries per tile); the
 * cull then scans all tiles.  Diagnostic only. */
typedef struct {
  int32_t nx, ny;
  int64_t entries;
  float x0, y0, cell, reach;
  float inv_cell; /* the FP32 1 / cell the kernels scale coordinates by */
} psdf_cull_grid_info;
int psdf_scene_cull_grid(const psdf_scene *scene, psdf_cull_grid_info *info);

/* Copies the cull grid's lists to the host (synchronous): offsets HOST
 * int32[nx * ny + 1] (cell c lists tiles[offsets[c] .. offsets[c + 1])),
 * tiles HOST int32[entries]; and every tile's AABB, aabbs HOST
 * float[n_tiles][4] (xmin, ymin, xmax, ymax), nullable.  Diagnostic only. */
int psdf_scene_cull_grid_copy(const psdf_scene *scene, int32_t *offsets, int32_t *tiles,
                              float *aabbs);

#define PSDF_MLP_IN 16
#define PSDF_MLP_HIDDEN 64
#define PSDF_PROPOSE_BOUND 1
#define PSDF_PROPOSE_MLP 2
#define PSDF_PROPOSE_CIRCLES 3
#define PSDF_CULL_MAX_K 4

typedef struct {
  int32_t mode; /* PSDF_PROPOSE_BOUND, PSDF_PROPOSE_MLP or PSDF_PROPOSE_CIRCLES */
  int32_t k;    /* proposals per pose, 1..PSDF_CULL_MAX_K (unused by PSDF_PROPOSE_CIRCLES) */
} psdf_cull_opts;

typedef struct {
  int64_t evaluated_obstacles; /* obstacles evaluated exactly (not skipped)       */
  int64_t evaluated_edges;     /* their edges                                     */
  int64_t proposed_items;      /* (pose, tile) pairs listed from the proposals    */
  int64_t fallback_items;      /* (pose, tile) pairs added by the bound check     */
  int64_t fallback_poses;      /* poses with at least one tile beyond the proposal */
  int64_t bound_evaluations;   /* tile lower bounds computed by the proposals     */
  int64_t circle_evaluations;  /* obstacle circles behind the upper bounds        */
} psdf_cull_stats;

/* Tile-proposal network: 16 inputs -> 64 ReLU units -> 1 output, FP16 weights
 * with FP32 accumulation (tensor-core mma).  W1 HOST float[64][16] row-major
 * (the hidden bias is the weight of input 15, which is the constant 1), w2
 * HOST float[64], b2 scalar; the weights are rounded to FP16 on upload. */
int psdf_mlp_create(const float *W1, const float *w2, float b2, psdf_mlp **out);
int psdf_mlp_destroy(psdf_mlp *mlp);

/* The network's inputs for (pose p, tile t), float[P][n_tiles][16] (DEVICE):
 * 0..7  the tile AABB corners (xmin,ymin) (xmax,ymin) (xmax,ymax) (xmin,ymax)
 *       in the pose frame, clamped to [-20, 20] m, times 0.1
 * 8..11 the corners' distances to p, clamped to [0, 30] m, times 0.1
 * 12    the distance from p to the AABB, clamped to [0, 30] m, times 0.1
 * 13    the footprint radius max_l |v_l| (m)
 * 14    the tile's edge count / 256
 * 15    1 */
int psdf_tile_features(const float *footprint, int32_t m, const psdf_scene *scene,
                       const float *poses, int64_t P, float *features, void *stream);

/* Network outputs (predicted signed distance of the tile's nearest obstacle)
 * for every (pose, tile), float[P][n_tiles] (DEVICE). */
int psdf_mlp_scores(const psdf_mlp *mlp, const float *footprint, int32_t m,
                    const psdf_scene *scene, const float *poses, int64_t P, float *scores,
                    void *stream);

/* Exact per-tile minimum signed distance for every (pose, tile),
 * float[P][n_tiles] (DEVICE): the training labels of the network. */
int psdf_tile_values(const float *footprint, int32_t m, const psdf_scene *scene,
                     const float *poses, int64_t P, const psdf_params *params, float *values,
                     void *stream);

/* The cull's bound LB (metres) for every (pose, tile), float[P][n_tiles]
 * (DEVICE).  LB > 0 proves that every obstacle of the tile is separated from
 * the posed footprint by more than LB; LB <= 0 makes no claim. */
int psdf_tile_lower_bounds(const float *footprint, int32_t m, const psdf_scene *scene,
                           const float *poses, int64_t P, float *lb, void *stream);

size_t psdf_cull_workspace_bytes(int64_t P, const psdf_scene *scene);

/* dphi and active are nullable; mlp may be NULL except for PSDF_PROPOSE_MLP. */
int psdf_eval_culled(const float *footprint, int32_t m, const psdf_scene *scene,
                     const psdf_mlp *mlp, const psdf_cull_opts *opts, const float *poses,
                     int64_t P, const psdf_params *params, float *phi, float *dphi,
                     uint32_t *active, void *workspace, size_t workspace_bytes, void *stream);
/* The same plus the saved backward records of psdf_backward_saved (see
 * there; hard minimum only). */
int psdf_eval_culled_save(const float *footprint, int32_t m, const psdf_scene *scene,
                          const psdf_mlp *mlp, const psdf_cull_opts *opts, const float *poses,
                          int64_t P, const psdf_params *params, float *phi, float *dphi,
                          uint32_t *active, float *saved, void *workspace,
                          size_t workspace_bytes, void *stream);

/* Synchronizes `stream` and copies the counters of the last psdf_eval_culled
 * that used `workspace` (PSDF_ERR_TIMEOUT if it recorded a device failure). */
int psdf_cull_stats_read(const void *workspace, void *stream, psdf_cull_stats *stats);

/* ---- training the tile-proposal network on the GPU ----------------------
 * Model s = w2 . relu(W1 x) + b2 (the network above, FP32 during training),
 * loss = mean over rows of (s - y)^2 where y is a clamped exact tile value
 * (psdf_tile_values).  Parameters are laid out as one float[1089] vector:
 * W1 row-major [64][16] | w2 [64] | b2.  Gradients are reduced in a fixed
 * order without atomics, so every step is reproducible bit for bit.
 * X DEVICE float[rows][16], y DEVICE float[rows]; idx (DEVICE int32[N],
 * nullable) selects the N rows of a step (NULL = the first N rows).
 * loss (DEVICE float, nullable) receives the step's mean loss before the
 * update.  Optimizer: Adam (0.9, 0.999, 1e-8) with bias correction. */
#define PSDF_MLP_PARAMS 1089
typedef struct psdf_trainer psdf_trainer;
int psdf_trainer_create(const float *W1, const float *w2, float b2, float lr,
                        psdf_trainer **out);
int psdf_trainer_destroy(psdf_trainer *trainer);
int psdf_trainer_set_lr(psdf_trainer *trainer, float lr);
/* gradient of the loss over rows 0..N-1 into DEVICE float[1089] */
int psdf_trainer_grad(psdf_trainer *trainer, const float *X, const float *y, int64_t N,
                      float *grad, float *loss, void *stream);
/* one Adam step on the rows idx[0..N-1] (or 0..N-1) */
int psdf_trainer_step(psdf_trainer *trainer, const float *X, const float *y, const int32_t *idx,
                      int64_t N, float *loss, void *stream);
/* state for checkpoints (HOST float[1089] each, nullable on get); both
 * synchronize the device */
int psdf_trainer_get(const psdf_trainer *trainer, float *params, float *m, float *v,
                     int64_t *step);
int psdf_trainer_set(psdf_trainer *trainer, const float *params, const float *m, const float *v,
                     int64_t step);

/* ---- batched plan: many instances in one persistent launch ---------------
 * Batching of MPC instances, SQP iterates and rollouts (Sec. IV-B, the
 * horizon stacked into one tensor, and Sec. V: per-stage edge sets E_{k+s}):
 * an INSTANCE is one footprint, one obstacle edge set of its own and a run of
 * poses.  Instances may differ in footprint size (3..16), edge count and
 * number of poses.  psdf_plan_create prepares every instance's scene once
 * (as psdf_scene_create_csr does) and lays all of them out in one device
 * image; psdf_eval_batched then evaluates every pose of every instance
 * against its own instance's edges (value, active pair, gradient -- the same
 * results psdf_eval_grad gives per instance, bit for bit) in ONE persistent
 * kernel launch: CTAs take work items (instance, block of its poses, run of
 * its edge tiles) from an atomic queue, largest first, and the CTA that
 * finishes the last item of a pose block runs that block's epilogue.
 *
 * Layout (all HOST pointers, copied at creation):
 *   footprints  float[sum m_i][2], instance i's footprint at vertex
 *               fp_offsets[i] .. fp_offsets[i+1]-1 (CCW, 3..16 vertices)
 *   edges       float[R][4] edge rows of all instances (Ax, Ay, Bx, By)
 *   obs_offsets int32[n_obs+1], CSR over the rows: obstacle q has rows
 *               obs_offsets[q] .. obs_offsets[q+1]-1 (1 edge = segment, >= 3
 *               = closed CCW convex polygon, as for psdf_scene_create_csr)
 *   inst_obs    int32[n_inst+1]: instance i owns obstacles inst_obs[i] ..
 *               inst_obs[i+1]-1, i.e. rows obs_offsets[inst_obs[i]] ..
 *               obs_offsets[inst_obs[i+1]]-1 (may be none)
 *   pose_offsets int64[n_inst+1]: instance i owns poses pose_offsets[i] ..
 *               pose_offsets[i+1]-1 of the pose array given to each call
 *   tile_edges  edges per tile (0 = 256; PSDF_TILE_MORTON selects Morton
 *               packing), as for scenes.
 * Active pair ids use the row index WITHIN the instance (row minus the
 * instance's first row).  params->eta > 0 selects the soft minimum for the
 * whole plan (evaluation, stage parameters and backward).
 *
 * The plan owns its device memory (scene image, work queue, per-pose keys).
 * psdf_eval_batched allocates nothing and never synchronizes: it issues two
 * memsets and one kernel on `stream`, so it can be captured in a CUDA graph.
 * Calls on one plan whose kernels overlap on the GPU race on its workspace
 * and must be serialized by the caller.
 *
 * Tile shapes: `threads` (CTA size 128 or 256; a pose block holds at most
 * `threads` poses, whose lanes split the tile's obstacles when fewer poses
 * than lanes are given) and `tiles_per_item` (edge tiles per work item,
 * 1..64).  psdf_plan_autotune times a grid of candidates on the caller's
 * poses (it synchronizes and allocates scratch: never call it during
 * capture), keeps the fastest, and caches the choice per plan shape (the
 * instances' pose, tile and footprint sizes on the current device) for the
 * life of the process; *from_cache (optional) reports a cache hit. */
typedef struct psdf_plan psdf_plan;

typedef struct {
  int32_t threads;
  int32_t tiles_per_item;
} psdf_plan_config;

typedef struct {
  int32_t n_inst;
  int32_t n_tiles;     /* edge tiles over all instances */
  int64_t n_poses;
  int64_t n_rows;      /* edge rows over all instances */
  int32_t n_items;     /* work items of the current configuration */
  int32_t n_blocks;    /* pose blocks of the current configuration */
  int32_t grid;        /* persistent CTAs launched */
  int32_t reserved;
  psdf_plan_config config;
  size_t device_bytes;
} psdf_plan_info;

int psdf_plan_create(int32_t n_inst, const float *footprints, const int32_t *fp_offsets,
                     const float *edges, const int32_t *obs_offsets, const int32_t *inst_obs,
                     const int64_t *pose_offsets, int32_t tile_edges, const psdf_params *params,
                     void *stream, psdf_plan **out);
int psdf_plan_destroy(psdf_plan *plan);
int psdf_plan_get_info(const psdf_plan *plan, psdf_plan_info *info);
/* Rebuilds the work queue for `config` (synchronizes the stream). */
int psdf_plan_set_config(psdf_plan *plan, const psdf_plan_config *config, void *stream);
int psdf_plan_autotune(psdf_plan *plan, const float *poses, int32_t reps, void *stream,
                       psdf_plan_config *chosen, int32_t *from_cache);
/* phi float[n_poses]; dphi float[n_poses][3] or NULL; active uint32[n_poses]
 * or NULL.  A bounded device wait that ran out turns the outputs of the pose
 * blocks finished after it into NaN; psdf_plan_status then reports
 * PSDF_ERR_TIMEOUT. */
int psdf_eval_batched(psdf_plan *plan, const float *poses, float *phi, float *dphi,
                      uint32_t *active, void *stream);
/* Stage parameters of every pose of a plan (time-varying edge sets: one
 * instance per stage, each with its own edges), as psdf_stage_params:
 * stage float[n_poses][4] = {phi - d_min, -d phi / d x}. */
int psdf_stage_params_batched(psdf_plan *plan, const float *poses, float d_min, float *stage,
                              uint32_t *active, void *stream);
/* Debug builds of the library (compiled with PSDF_DEBUG_CHECKS) check every
 * index the batched kernels take from their data before using it, record
 * the first violation as (site << 48 | index) and skip the access; this
 * returns that record (0 = none) and *enabled = 1.  Release builds return
 * *enabled = 0 and *violation = 0. */
int psdf_plan_debug_read(uint64_t *violation, int32_t *enabled);
/* Synchronizes the stream and reports whether the last psdf_eval_batched
 * met a timed-out wait. */
int psdf_plan_status(const psdf_plan *plan, void *stream);
/* Vector-Jacobian product through each pose's active pair, as psdf_backward
 * per instance: grad_pose float[n_poses][3] (written, or NULL), grad_edges
 * float[R][4] over all instances' rows (accumulated with atomics, or NULL). */
int psdf_backward_batched(const psdf_plan *plan, const float *poses, const uint32_t *active,
                          const float *grad_phi, float *grad_pose, float *grad_edges,
                          void *stream);

/* ---- value + gradient without any device allocation ---------------------
 * The paper has no counterpart: this serves callers that cannot allocate
 * device memory while they run -- a control loop with a hard period (an
 * allocation may synchronize the device and stall it), a plug-in whose host
 * framework owns the whole memory pool, code running where the allocator is
 * locked.  It computes exactly what psdf_eval_grad computes (same inputs,
 * outputs, kernels and results) but takes its scratch from a fixed device
 * array built into the library instead of a caller workspace, and it calls no
 * cudaMalloc, cudaFree or other allocating routine.
 *  - The array holds PSDF_NOALLOC_MAX_POSES keys (2 MiB + 256 bytes); every
 *    GPU that loads the library keeps it until the process exits.  P above
 *    the maximum is rejected with PSDF_ERR_CAPACITY.
 *  - The first call on a device looks up the array's device address (once,
 *    with that device current, and again after the device's context was
 *    replaced, e.g. by cudaDeviceReset); make that first call before any
 *    stream capture.
 *  - Every call shares the one array: calls whose kernels overlap on the GPU
 *    (other streams, other threads) race and must be serialized by the
 *    caller.  Each call re-initializes the scratch it uses, so the previous
 *    call's contents never leak into its results.
 *  - The error word lives in the built-in array, which psdf_workspace_status
 *    cannot read: a device-side wait that ran out shows only in the outputs
 *    (phi = NaN, dphi = NaN, active = PSDF_PAIR_NONE for the affected
 *    poses). */
#define PSDF_NOALLOC_MAX_POSES 262144
int psdf_eval_grad_noalloc(const float *footprint, int32_t m, const psdf_scene *scene,
                           const float *poses, int64_t P, const psdf_params *params, float *phi,
                           float *dphi, uint32_t *active, void *stream);

/* ---- failure detection (for tests) ---------------------------------------
 * The library has no counterpart in the paper here.  Its only device-side
 * waits are the bounded mbarrier waits for the tile copies of the full scan
 * (psdf_eval, psdf_eval_grad, psdf_stage_params, the no-allocation call) and
 * of the batched plans; each gives up after `polls` polls (default 4194304,
 * i.e. 1 << 22), records the failure (psdf_workspace_status /
 * psdf_plan_status then report PSDF_ERR_TIMEOUT) and turns the affected
 * poses' outputs into phi = NaN, dphi = NaN, active = PSDF_PAIR_NONE.  This
 * sets the limit for every launch issued afterwards in the process (a CUDA
 * graph keeps the limit it was captured with); 0 makes every such wait give
 * up at once, which drives that path without any fault or hang: a kernel
 * whose wait gave up still waits, with the default limit, for the copies it
 * has issued before it exits.  The exact tile cull has no device-side wait.
 * *previous (nullable) receives the limit that was in force. */
int psdf_debug_set_wait_limit(uint32_t polls, uint32_t *previous);

/* ---- measurement --------------------------------------------------------
 * No counterpart in the paper: the FP32 roofline's denominator, measured.
 * Runs an FP32 FMA microbenchmark on the current device (every SM full of
 * threads running 8 independent multiply-add chains each, `iters` steps,
 * scalar FMAs or, paired != 0, paired FP32 FMAs on float2) reps + 1 times on
 * `stream` (the first launch warms up), synchronously, and returns the best
 * rate in TFLOP/s (2 flops per FMA) and its duration.  It allocates a small
 * output buffer and synchronizes: never call it during stream capture. */
int psdf_measure_fp32_peak(int32_t paired, int32_t iters, int32_t reps, double *tflops,
                           double *best_ms, void *stream);

/* ---- tracing -----------------------------------------------------------
 * When enabled, the library brackets each launch of its kernels with CUDA
 * events recorded on the launch stream (not during stream capture).
 * psdf_profile_read synchronizes those events and returns, for the kernel
 * named `kernel` ("scan", "epilogue", "backward", "all"), the number of
 * launches and their summed device time since the last reset.  Names that
 * match no kernel report zero launches. */
int psdf_profile_enable(int on);
int psdf_profile_reset(void);
int psdf_profile_read(const char *kernel, int64_t *launches, double *total_ms);

#ifdef __cplusplus
}
#endif

#endif /* PSDF_H */
