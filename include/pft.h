/*
 * pft.h -- C ABI of libpft: direct (non-FFT) Fourier transform of polygonal
 * areas and of closed surfaces of triangles or planar polygons, one shape or
 * batches of many, with adjoints, on one NVIDIA GB300 (sm_103a).
 *
 * Method: B. B. Maranville, "An implementation of an efficient direct Fourier
 * transform of polygonal areas and volumes", arXiv 2104.08309.
 *   FT(Q) = integral over the region of exp(+i Q.r) dA (2D) or dV (3D)  (Sec. 2, Sec. 3 Eq. 7)
 * evaluated by the divergence theorem (Eq. 1, Eq. 8) as a sum over boundary
 * segments (2D, Eq. 6) or over faces and their edges (3D, Eq. 14 with the overall
 * sign fixed so that FT(0) = +volume for outward faces).  Q carries no 2 pi.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Every array argument is a DEVICE pointer owned by the caller.  The library
 *    never allocates or frees device memory in these calls; scratch space comes
 *    from the caller as `ws` (at least `*_workspace_size` bytes, 256-byte aligned).
 *  - Calls only enqueue work on `stream` (a cudaStream_t passed as void*; NULL =
 *    the legacy default stream) and return at once.  Argument errors are
 *    returned synchronously; errors the GPU detects (bad index, non-finite
 *    coordinate, malformed offsets, a wait that timed out) are written into a
 *    status word inside `ws`, read back with pft_status().
 *  - Vertices are float32 and are taken as exact.  Q is float64 at the boundary;
 *    the FP32 path rounds it once on the device.  Outputs are float64 (re, im)
 *    pairs and are fully overwritten.
 *  - Results are deterministic: no floating-point atomics; every reduction runs
 *    in a fixed order.
 *  - Thread safety: no mutable global state apart from the fixed scratch of
 *    pft3d_mesh_noalloc (see there) and per-thread launch counters; concurrent
 *    calls need separate workspaces.
 */
#ifndef PFT_H
#define PFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes (synchronous) and status-word values (device-detected). */
typedef enum {
  PFT_OK = 0,
  PFT_ERR_INVALID_ARG = 1,   /* null pointer, negative count, bad option          */
  PFT_ERR_INDEX_RANGE = 2,   /* face index outside [0, n_verts) (status word)     */
  PFT_ERR_NONFINITE = 3,     /* NaN/Inf vertex coordinate (status word)           */
  PFT_ERR_WORKSPACE = 4,     /* ws NULL, misaligned or smaller than required      */
  PFT_ERR_CUDA = 5,          /* a CUDA launch or copy failed                      */
  PFT_ERR_TIMEOUT = 6,       /* a bounded wait on a copy gave up (status word)    */
  PFT_ERR_UNSUPPORTED = 7,   /* option combination not implemented                */
  PFT_ERR_OFFSETS = 8,       /* CSR offsets not non-decreasing / inconsistent     */
  PFT_ERR_SCRATCH_LIMIT = 9, /* problem too large for pft3d_mesh_noalloc's scratch */
  PFT_ERR_PAIRS = 10         /* faces given as pairs do not share their first edge (status word) */
} pft_status_code;

typedef enum {
  PFT_FP32_COMPENSATED = 0,  /* FP32 bulk arithmetic, compensated sums, FP64 finish */
  PFT_FP64 = 1               /* plain FP64 throughout (comparison path)             */
} pft_precision;

typedef enum {
  PFT_Q_TILED = 0,           /* the main kernel visits Q points in the library's order */
  PFT_Q_AS_GIVEN = 1         /* ... in the caller's order                              */
} pft_q_order_mode;

/*
 * Options.  Zero-initialised means "defaults".  A NULL pointer is the same as
 * all defaults.
 *  precision        pft_precision.
 *  q_per_thread     Q points each thread keeps in registers (0 = default; FP32: 1, 2,
 *                   4 or 8; FP64: 1 or 2).
 *  block_threads    threads per block of the main kernel (0 = default; 128 or 256; the
 *                   batched FP32 calls also take 512 with q_per_thread 4, one block per SM,
 *                   and take it by default on a shared Q set of 4 x 512 points or more).
 *  k_splits         number of segment/face chunks summed in the FP64 second pass
 *                   (0 = chosen from the problem size and the GPU).  For a fixed
 *                   value and launch shape the result is bitwise reproducible;
 *                   different values agree to rounding.
 *  tile_items       must be 0 (the shared-memory tile size is fixed per path).
 *  face_series_tau  3D only: faces whose corner phases satisfy
 *                   P = (a0^2 + a1^2 + a2^2)/2 < tau^2/4 (a_k = Q.(p_k - centroid);
 *                   this implies max_l |Q.d_l| < tau) take the series of the face
 *                   integral (Eq. 13) instead of the edge sum of Eq. 14, which
 *                   cancels there.  The decision is made per face for each group
 *                   of 32 threads' Q points; a group whose P are all below 1/4
 *                   takes a short form of the series, one with P up to 9/4 a
 *                   longer form, one with P up to 9 the longest.  Must lie in
 *                   (0, 6]; 0 = default 6.0 (fewest operations per pair; 1.0
 *                   keeps the edge sum for every face whose spread is at least
 *                   1, where it loses nothing to cancellation).  The FP64 path
 *                   uses at most 3.0 (its series is kept through k = 16).
 *  face_pairs       3D triangle calls (pft3d_mesh and its no-workspace form): the
 *                   number of leading face pairs.  For k < face_pairs, faces 2k
 *                   and 2k+1 must share their first edge in opposite directions,
 *                   (a, b, c) and (b, a, d), as pft3d_pair_faces writes them; the
 *                   FP32 path then evaluates that edge's sinc(Q.d/2) once for both
 *                   faces where a group of 32 threads takes the edge sum of Eq. 14
 *                   for both.  The device checks every pair (a pair that does not
 *                   share its first edge contributes nothing and sets
 *                   PFT_ERR_PAIRS).  0 = no pairs; 2 face_pairs <= n_faces.  Other
 *                   calls ignore it.
 *  q_order          forward calls (pft2d_polygons, pft3d_mesh, pft3d_polymesh, the
 *                   no-workspace form, and the batched calls on a shared Q set):
 *                   PFT_Q_TILED (0, default) lets the library choose the order in
 *                   which the main kernel visits the Q points.  It sorts them along
 *                   a Z-order curve of their coordinates (quantised over their
 *                   bounding box) and gives each group of 32 threads a run of nearby
 *                   points, because the 3D series-or-edge-sum choice and the 2D SFU
 *                   sinc are decided per group.  It does so only when there are at
 *                   least two blocks' worth of Q points and about 1e9 pairs or more.
 *                   PFT_Q_AS_GIVEN (1) keeps the caller's order.  Outputs are in the
 *                   caller's order either way.  The two agree bitwise in 2D and to
 *                   rounding in 3D (another grouping can switch a face between the
 *                   series and the edge sum for some Q points).  Other values:
 *                   PFT_ERR_INVALID_ARG.
 *  main_start_event, main_stop_event
 *                   cudaEvent_t handles or NULL.  When set, they are recorded on
 *                   `stream` immediately before and after the main pair kernel
 *                   (the pair sum of a forward call, the pair adjoint of a
 *                   backward or Q-gradient call), so that a caller can time it
 *                   alone.
 */
typedef struct {
  int32_t precision;
  int32_t q_per_thread;
  int32_t block_threads;
  int32_t k_splits;
  int32_t tile_items;
  float face_series_tau;
  void* main_start_event;
  void* main_stop_event;
  int32_t face_pairs;
  int32_t q_order;
  int32_t reserved[2];
} pft_options;

/* Bytes of workspace the matching call needs for these sizes and options. */
size_t pft2d_workspace_size(int64_t n_verts, int64_t n_loops, int64_t n_q, const pft_options* opts);
size_t pft3d_workspace_size(int64_t n_verts, int64_t n_faces, int64_t n_q, const pft_options* opts);

/*
 * 2D: FT_A(Q) of the region bounded by closed loops (Sec. 2, Eq. 6 per segment).
 *  verts     [n_verts][2] float32.  Loop l is verts[loop_off[l] .. loop_off[l+1]-1],
 *            its last vertex joined to its first.  CCW loops add area, CW loops
 *            subtract it (holes).
 *  loop_off  [n_loops+1] int64, loop_off[0] = 0, non-decreasing,
 *            loop_off[n_loops] = n_verts (checked on the device -> PFT_ERR_OFFSETS).
 *  q         [n_q][2] float64.      out  [n_q][2] float64 (re, im).
 */
int pft2d_polygons(const float* verts, int64_t n_verts, const int64_t* loop_off, int64_t n_loops,
                   const double* q, int64_t n_q, double* out,
                   void* ws, size_t ws_bytes, const pft_options* opts, void* stream);

/*
 * Batched 2D: one FT_A per polygon (Sec. 2, Eq. 6 per segment), thousands of
 * polygons of uneven sizes in one persistent launch.  Two steps:
 *
 * 1. pft2d_batched_prepare (host work + copies; synchronises `stream`; not for
 *    use inside stream capture): cuts every polygon into work items (polygon,
 *    segment chunk of <= 4096, Q tile), sorts them by cost and deals them to the
 *    persistent blocks longest-first onto the least-loaded block, then copies that
 *    static schedule into `ws` and fills `plan` (a small host struct the caller
 *    keeps).  Redo it whenever the offsets, n_q or the options change.
 * 2. pft2d_polygons_batched (kernel launches only, so a CUDA graph can capture
 *    and replay it): runs the prepared schedule on the current vertices and Q.
 *
 *  verts        [n_verts][2] float32; polygon i is one CCW loop
 *               verts[poly_off[i] .. poly_off[i+1]-1].
 *  poly_off     [n_polys+1] int64: HOST copy for prepare, DEVICE copy for the call
 *               (the device checks that it matches the plan -> PFT_ERR_OFFSETS).
 *  q, q_off     float64 Q points.  With q_off == NULL every polygon uses all n_q
 *               points and out is [n_polys][n_q][2]; otherwise polygon i uses
 *               q[q_off[i] .. q_off[i+1]-1] and out is [n_q][2] in the same order
 *               (q_off: HOST copy for prepare, DEVICE copy for the call).
 *  opts         precision, q_per_thread, block_threads, q_order (shared Q set only:
 *               per-polygon Q lists keep their order) (k_splits, tile_items 0).
 * Workspace size from pft2d_batched_workspace_size (same host arguments).
 */
typedef struct {
  int64_t opaque[24];
} pft_batched_plan;

size_t pft2d_batched_workspace_size(int64_t n_verts, const int64_t* poly_off_host, int64_t n_polys,
                                    const int64_t* q_off_host, int64_t n_q, const pft_options* opts);
int pft2d_batched_prepare(const int64_t* poly_off_host, int64_t n_polys, const int64_t* q_off_host, int64_t n_q,
                          void* ws, size_t ws_bytes, const pft_options* opts, pft_batched_plan* plan,
                          void* stream);
int pft2d_polygons_batched(const float* verts, int64_t n_verts, const int64_t* poly_off, int64_t n_polys,
                           const double* q, const int64_t* q_off, int64_t n_q, double* out,
                           void* ws, size_t ws_bytes, const pft_batched_plan* plan, void* stream);

/*
 * Batched 3D: one FT_V per closed triangle mesh, for many meshes of uneven size,
 * in one persistent launch (the same design as the batched 2D calls above).
 *  verts     [n_verts][3] float32, shared by all meshes.
 *  faces     [n_faces][3] int32 indices into verts, each triangle counter-
 *            clockwise seen from outside its mesh.
 *  mesh_off  [n_meshes + 1] int64 (CSR over faces): mesh i is faces
 *            mesh_off[i] .. mesh_off[i+1]-1.  The host copy given to
 *            pft3d_batched_prepare and the device copy given to
 *            pft3d_meshes_batched must hold the same values.
 *  q, q_off, out   as for pft2d_polygons_batched, with 3 coordinates per Q.
 * Options as for pft3d_mesh (face_series_tau included); launch shapes: FP32
 * 2 or 4 Q points per thread with 128 threads (default 4), FP64 1 with 128.
 * The plan from pft3d_batched_prepare is only valid for pft3d_meshes_batched.
 */
size_t pft3d_batched_workspace_size(int64_t n_faces, const int64_t* mesh_off_host, int64_t n_meshes,
                                    const int64_t* q_off_host, int64_t n_q, const pft_options* opts);
int pft3d_batched_prepare(const int64_t* mesh_off_host, int64_t n_meshes, const int64_t* q_off_host, int64_t n_q,
                          void* ws, size_t ws_bytes, const pft_options* opts, pft_batched_plan* plan,
                          void* stream);
int pft3d_meshes_batched(const float* verts, int64_t n_verts, const int32_t* faces, int64_t n_faces,
                         const int64_t* mesh_off, int64_t n_meshes, const double* q, const int64_t* q_off,
                         int64_t n_q, double* out, void* ws, size_t ws_bytes, const pft_batched_plan* plan,
                         void* stream);

/* Kernel launches enqueued by the most recent batched call (2D or 3D) on this host thread. */
int pft_batched_last_launch_count(void);

/*
 * 3D: FT_V(Q) of a closed surface of triangles (Sec. 3, Eq. 14 sign-corrected).
 *  verts  [n_verts][3] float32.
 *  faces  [n_faces][3] int32, 0-based, each triangle counter-clockwise seen from
 *         outside (outward normal).  Out-of-range indices set PFT_ERR_INDEX_RANGE
 *         and the face is skipped.
 *  q      [n_q][3] float64.      out  [n_q][2] float64 (re, im).
 */
int pft3d_mesh(const float* verts, int64_t n_verts, const int32_t* faces, int64_t n_faces,
               const double* q, int64_t n_q, double* out,
               void* ws, size_t ws_bytes, const pft_options* opts, void* stream);

/*
 * Host helper for the face_pairs option (Sec. 3, Eq. 14: on a closed surface every
 * edge belongs to two faces, and its sinc(Q.d/2) is the same for both, since sinc
 * is even and d only flips sign).  Reorders a triangle list so that as many faces
 * as possible come in pairs that share an edge: faces_out[2k], faces_out[2k+1] =
 * (a, b, c), (b, a, d) for k < *n_pairs, then the faces left unpaired in their
 * input order and vertex order.  Pairs join faces that hold a common edge in
 * opposite directions (an edge of more than two faces, or of two faces in the
 * same direction, pairs nothing), chosen by a deterministic Karp-Sipser matching:
 * a face with one free neighbour is matched to it first, else the lowest-numbered
 * free face to its first free neighbour (about 98 % of an icosphere's faces end
 * up in pairs; O(n) time and memory on the host).  The result
 * describes the same surface (a rotation of a triangle's corners keeps it), so
 * every transform of it is unchanged.
 *  faces_host  [n_faces][3] int32, HOST memory, indices >= 0.
 *  faces_out   [n_faces][3] int32, HOST memory, written (may not alias faces_host).
 *  n_pairs     receives the number of pairs.
 * Returns PFT_OK, PFT_ERR_INVALID_ARG (null pointer, negative count or index).
 * Synchronous host work; no GPU is touched.
 */
int pft3d_pair_faces(const int32_t* faces_host, int64_t n_faces, int32_t* faces_out, int64_t* n_pairs);

/*
 * The Q order of the q_order option (PFT_Q_TILED) as a slot -> Q index map, for a
 * caller that wants to see it or reuse it.  The main kernel with q_per_thread Q
 * points per thread and block_threads threads per block visits Q point perm[s] in
 * slot s, and the slots base + r*block_threads + 32*w + lane (r < q_per_thread,
 * lane < 32) of a block form group w of 32 threads.  The Q points are sorted along
 * a Z-order curve of their FP32 coordinates, quantised over their bounding box
 * (10 bits per axis in 3D, 16 in 2D; NaN coordinates count as the lowest level),
 * by a stable radix sort, and each run of 32 q_per_thread sorted points fills one
 * group's slots; the last, partial block keeps the sorted order.
 *  q          [n_q][dim] float64, device.      perm  [n_q] int32, device, written.
 *  dim        2 or 3; q_per_thread 1, 2, 4 or 8; block_threads 128, 256 or 512.
 * Workspace: pft_q_order_workspace_size(n_q) bytes, 256-byte aligned.
 * Returns PFT_OK, PFT_ERR_INVALID_ARG, PFT_ERR_UNSUPPORTED (n_q > INT32_MAX or
 * another shape), PFT_ERR_WORKSPACE, PFT_ERR_CUDA.  Asynchronous on `stream`.
 */
size_t pft_q_order_workspace_size(int64_t n_q);
int pft_q_order(const double* q, int64_t n_q, int dim, int q_per_thread, int block_threads, int32_t* perm, void* ws,
                size_t ws_bytes, void* stream);

/*
 * 3D: FT_V(Q) of a closed surface of planar polygon faces of any size (Sec. 3:
 * Eq. 14 is stated for polygon faces and their edges).
 *  face_idx  [n_idx] int32, 0-based vertex indices of all faces, concatenated;
 *            each face counter-clockwise seen from outside, planar, at least 3
 *            vertices; non-convex faces are allowed.
 *  face_off  [n_faces + 1] int64 on the device: face m is
 *            face_idx[face_off[m] .. face_off[m+1]-1]; face_off[0] = 0 and
 *            face_off[n_faces] = n_idx.  Malformed offsets set PFT_ERR_OFFSETS.
 *  The device splits every face into n - 2 triangles by recursive halving (the
 *  chain p_i .. p_j becomes the triangle (p_i, p_m, p_j), m = (i + j)/2, and
 *  the chains p_i .. p_m and p_m .. p_j, from p_0 .. p_{n-1}), which tile a
 *  planar polygon with signed areas, so the result is the same integral, and
 *  whose interior diagonals stay short (their terms cancel only up to
 *  rounding); then it runs the pft3d_mesh path on the n_idx - 2 n_faces
 *  triangles (same options).  n_idx >= 3 n_faces is required.
 */
size_t pft3d_polymesh_workspace_size(int64_t n_verts, int64_t n_idx, int64_t n_faces, int64_t n_q,
                                     const pft_options* opts);
int pft3d_polymesh(const float* verts, int64_t n_verts, const int32_t* face_idx, int64_t n_idx,
                   const int64_t* face_off, int64_t n_faces, const double* q, int64_t n_q, double* out,
                   void* ws, size_t ws_bytes, const pft_options* opts, void* stream);

/*
 * Backward passes: adjoints of pft2d_polygons / pft3d_mesh with respect to the
 * vertices (the paper has no gradients; they differentiate its sums, Eq. 6 and
 * Eq. 14, term by term).
 *  grad_out   [n_q][2] float64: (dL/dRe F, dL/dIm F) at each Q.
 *  grad_verts [n_verts][d] float32: dL/dverts = sum_Q Re(conj(g_Q) dF(Q)/dverts),
 *             g_Q = grad_out[Q][0] + i grad_out[Q][1].  Overwritten.
 * Segment/face terms are recomputed (not stored by the forward call) and
 * differentiated in reverse mode exactly as the FP32 forward evaluates them, in
 * FP32 with compensated sums; Q = 0 and |Q| max|r - c| < 0.25 use an FP64
 * boundary-flux series instead.  Options: precision must be
 * PFT_FP32_COMPENSATED; launch fields 0; face_series_tau as in the forward.
 * Vertex sums run in a fixed order (3D: through a device-built, sorted
 * vertex -> face-corner list), so results are reproducible.
 */
size_t pft2d_backward_workspace_size(int64_t n_verts, int64_t n_loops, int64_t n_q, const pft_options* opts);
size_t pft3d_backward_workspace_size(int64_t n_verts, int64_t n_faces, int64_t n_q, const pft_options* opts);
int pft2d_polygons_backward(const float* verts, int64_t n_verts, const int64_t* loop_off, int64_t n_loops,
                            const double* q, int64_t n_q, const double* grad_out, float* grad_verts,
                            void* ws, size_t ws_bytes, const pft_options* opts, void* stream);
int pft3d_mesh_backward(const float* verts, int64_t n_verts, const int32_t* faces, int64_t n_faces,
                        const double* q, int64_t n_q, const double* grad_out, float* grad_verts,
                        void* ws, size_t ws_bytes, const pft_options* opts, void* stream);

/* Adjoint of a batch of polygons, the backward of pft2d_polygons_batched: poly_off
 * [n_polys + 1] int64 on the device (each polygon one counter-clockwise loop;
 * malformed offsets set PFT_ERR_OFFSETS); Q as in the forward call: q_off == NULL
 * for one shared list of n_q points (grad_out [n_polys][n_q][2]), or q_off
 * [n_polys + 1] int64 on the device giving polygon i the points q[q_off[i] ..
 * q_off[i+1]-1] (grad_out [n_q][2] in the same order; malformed q_off sets
 * PFT_ERR_OFFSETS).  grad_out holds (dL/dRe F_i(Q), dL/dIm F_i(Q)); grad_verts
 * [n_verts][2] float32 is overwritten with sum_Q Re(conj(g_i) dF_i/dv) for the
 * vertices of polygon i.  The workspace holds one 36-byte Q record per (polygon,
 * Q) row (n_polys x n_q rows shared, n_q rows with q_off) plus per-vertex terms;
 * per_polygon_q tells the size function which (0: shared, 1: q_off). */
size_t pft2d_batched_backward_workspace_size(int64_t n_verts, int64_t n_polys, int64_t n_q, int per_polygon_q,
                                             const pft_options* opts);
int pft2d_polygons_batched_backward(const float* verts, int64_t n_verts, const int64_t* poly_off, int64_t n_polys,
                                    const double* q, const int64_t* q_off, int64_t n_q, const double* grad_out,
                                    float* grad_verts, void* ws, size_t ws_bytes, const pft_options* opts,
                                    void* stream);

/* Adjoint of a batch of closed triangle meshes, the backward of pft3d_meshes_batched:
 * verts [n_verts][3] float32 shared by all meshes, faces [n_faces][3] int32 (global
 * vertex indices), mesh_off [n_meshes + 1] int64 on the device (CSR over faces:
 * mesh i is faces mesh_off[i] .. mesh_off[i+1]-1; malformed offsets set
 * PFT_ERR_OFFSETS); Q as in the forward call: q_off == NULL for one shared list of
 * n_q points (grad_out [n_meshes][n_q][2]) or per-mesh lists q[q_off[i] ..
 * q_off[i+1]-1] (grad_out [n_q][2]).  grad_verts [n_verts][3] float32 is overwritten
 * with sum over meshes and their Q of Re(conj(g_i) dF_i/dv) (vertices used by no mesh
 * get 0).  Each mesh is centred on the bounding box of its own corners; the pair
 * adjoint is that of pft3d_mesh_backward (Eq. 14 and its series differentiated in
 * reverse mode, FP32 with compensated sums; |Q| r_max < 0.25 in FP64 from the corner
 * series), the vertex sums in a fixed order.  Options and errors as for
 * pft3d_mesh_backward; the workspace holds one 36-byte Q record per (mesh, Q) row
 * (n_meshes x n_q rows shared, n_q rows with q_off) plus 204 bytes per face.
 * per_mesh_q tells the size function which (0: shared, 1: q_off). */
size_t pft3d_batched_backward_workspace_size(int64_t n_verts, int64_t n_faces, int64_t n_meshes, int64_t n_q,
                                             int per_mesh_q, const pft_options* opts);
int pft3d_meshes_batched_backward(const float* verts, int64_t n_verts, const int32_t* faces, int64_t n_faces,
                                  const int64_t* mesh_off, int64_t n_meshes, const double* q, const int64_t* q_off,
                                  int64_t n_q, const double* grad_out, float* grad_verts, void* ws, size_t ws_bytes,
                                  const pft_options* opts, void* stream);

/* Adjoint of pft3d_polymesh (same faces, same split into triangles): grad_verts
 * [n_verts][3] float32 from grad_out as for pft3d_mesh_backward.  The workspace
 * must also hold the triangle list (see the size function). */
size_t pft3d_polymesh_backward_workspace_size(int64_t n_verts, int64_t n_idx, int64_t n_faces, int64_t n_q,
                                              const pft_options* opts);
int pft3d_polymesh_backward(const float* verts, int64_t n_verts, const int32_t* face_idx, int64_t n_idx,
                            const int64_t* face_off, int64_t n_faces, const double* q, int64_t n_q,
                            const double* grad_out, float* grad_verts, void* ws, size_t ws_bytes,
                            const pft_options* opts, void* stream);

/*
 * Q-gradient of a loss on FT_V (3D triangles): grad_q[n_q][3] float64 receives
 * dL/dQ = Re(conj(g_Q) dF(Q)/dQ) for grad_out as above.  Not in the paper; it
 * is the derivative of the forward sum (Eq. 14 and its series) with respect to
 * Q: dF/dQ = F (i c - 2Q/|Q|^2) + e^{iQ.c}/|Q|^2 dS/dQ, the last term from the
 * same reverse pass per (Q, face) pair as the vertex adjoint, accumulated per
 * Q instead of per face; Q = 0 and small |Q| in FP64 from the derivative of the
 * tetrahedron series.  Options and errors as for pft3d_mesh_backward.
 */
size_t pft3d_qgrad_workspace_size(int64_t n_verts, int64_t n_faces, int64_t n_q, const pft_options* opts);
int pft3d_mesh_qgrad(const float* verts, int64_t n_verts, const int32_t* faces, int64_t n_faces,
                     const double* q, int64_t n_q, const double* grad_out, double* grad_q,
                     void* ws, size_t ws_bytes, const pft_options* opts, void* stream);

/*
 * Q-gradient of a loss on FT_A (2D loops): grad_q[n_q][2] float64 receives
 * dL/dQ = Re(conj(g_Q) dF(Q)/dQ) for grad_out [n_q][2] as above.  Not in the
 * paper; the derivative of its segment sum (Sec. 2, Eq. 6) with respect to Q:
 * with F = e^{iQ.c} (2/|Q|^2) S and S = sum over segments of
 * -i w sinc(u) e^{i phi} (phi = Q.m, u = Q.h, w = Qx hy - Qy hx for the midpoint
 * m and half edge vector h, relative to the bounding-box centre c),
 *   dF/dQ = F (i c - 2Q/|Q|^2) + e^{iQ.c} (2/|Q|^2) dS/dQ,
 * the last term from the reverse pass of every (Q, segment) pair in FP32 with
 * compensated sums, accumulated per Q; Q = 0 and |Q| max|r - c| < 0.25 in FP64 from
 * the derivative of the fan-triangle series.  Arguments, options and errors as
 * for pft2d_polygons_backward (malformed loop_off sets PFT_ERR_OFFSETS).
 */
size_t pft2d_qgrad_workspace_size(int64_t n_verts, int64_t n_loops, int64_t n_q, const pft_options* opts);
int pft2d_polygons_qgrad(const float* verts, int64_t n_verts, const int64_t* loop_off, int64_t n_loops,
                         const double* q, int64_t n_q, const double* grad_out, double* grad_q,
                         void* ws, size_t ws_bytes, const pft_options* opts, void* stream);

/* Kernel launches enqueued by the most recent backward call on this host thread. */
int pft_backward_last_launch_count(void);

/*
 * pft3d_mesh without a workspace argument, for callers that cannot allocate
 * device memory when they need a transform: code running while a stream is
 * captured into a CUDA graph, plug-ins whose host application owns all device
 * allocations, loops that forbid allocation after start-up.  (The paper has no
 * counterpart; this is a calling convenience.)
 *  - Same arguments, result and options as pft3d_mesh, minus ws / ws_bytes.
 *    It allocates nothing and calls no allocating routine.
 *  - Scratch is a file-scope device array of 32 MiB, which every GPU that loads
 *    the library keeps until the process exits.  Problems whose
 *    pft3d_workspace_size() exceeds 32 MiB return PFT_ERR_SCRATCH_LIMIT at once.
 *  - All calls on a device share that array and it keeps the last call's
 *    contents; calls whose GPU work overlaps (several streams or host threads)
 *    race on it, so serialise them.
 *  - The first call on each device looks up the array's address (with that
 *    device current); make it before any stream capture begins.  Later calls
 *    made outside stream capture look it up again (so a context recreated after
 *    cudaDeviceReset is followed); a call inside a capture uses the address
 *    cached by the last call outside one, so do not reset the device between
 *    that call and the capture.
 *  - Sizes or options that pft3d_mesh rejects are rejected with the same code.
 *  - Device-detected input errors are recorded in the shared scratch, which
 *    callers cannot read: validate indices and coordinates beforehand, or use
 *    pft3d_mesh and pft_status() where that matters.
 */
int pft3d_mesh_noalloc(const float* verts, int64_t n_verts, const int32_t* faces, int64_t n_faces,
                       const double* q, int64_t n_q, double* out, const pft_options* opts, void* stream);

/*
 * Device-detected status of the last call that used `ws`: synchronises `stream`,
 * copies the status word back and returns PFT_OK or the first error found
 * (PFT_ERR_INDEX_RANGE, PFT_ERR_NONFINITE, PFT_ERR_OFFSETS, PFT_ERR_TIMEOUT), or
 * PFT_ERR_CUDA if the copy itself failed.
 */
int pft_status(const void* ws, void* stream);

/*
 * Self-test of the failure handling around the copies (no counterpart in the paper).
 * Every wait of the kernels on an mbarrier is bounded; when it runs out the kernel
 * sets the timeout bit of the status word in its workspace and returns, so the
 * context stays usable.  This call exercises that path: it clears the 256-byte
 * header at `ws` (device, 256-byte aligned, ws_bytes >= 256) and launches one block
 * that polls an mbarrier `polls` times (1 .. 2^20).  With arrive = 0 nothing
 * completes the barrier's phase, the wait runs out, and pft_status(ws) then returns
 * PFT_ERR_TIMEOUT; with arrive = 1 the block arrives first, the wait succeeds and
 * pft_status returns PFT_OK.  Errors: PFT_ERR_WORKSPACE (ws), PFT_ERR_INVALID_ARG
 * (polls, arrive), PFT_ERR_CUDA (launch).  Asynchronous on `stream`.
 */
int pft_selftest_wait(void* ws, size_t ws_bytes, uint32_t polls, int arrive, void* stream);

/* Static English text for a code (never NULL). */
const char* pft_status_string(int code);

/* Library version as 10000*major + 100*minor + patch. */
int pft_version(void);

/* Number of kernel launches the most recent call on this host thread enqueued (for accounting). */
int pft_last_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* PFT_H */
