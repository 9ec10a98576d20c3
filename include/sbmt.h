/*
 * sbmt.h -- C interface of the GB300 library for Structured Bitmap-to-Mesh
 * Triangulation (SBMT, arXiv 2602.19474).
 *
 * The library turns a label bitmap into a conforming triangle mesh: it
 * extracts the pixel-edge boundary of the labels (the "input boundary as
 * prescribed prior" of Sec. 3.1), overlays the regular equilateral base grid
 * of edge h (Sec. 3.3), classifies every segment/edge incidence by Alg. 1
 * (Sec. 3.3.1), keys each cut grid triangle by its canonical configuration
 * kappa(K) and replaces it by the patch of the single-valued lookup table
 * (Sec. 3.3.3, Alg. 2, App. G), and leaves every uncut grid triangle as it is.
 * All steps run in CUDA kernels on the GPU; there is no CPU fallback.
 *
 * Conventions
 *  - Every function returns an int: SBMT_OK (0) or a negative SBMT_E* code.
 *    No function throws, aborts or traps.
 *  - Pixels are unit squares centred at integer points; pixel (x, y) is
 *    data[y * pitch + x]; y grows with the row index and the mesh is
 *    counter-clockwise in that (x, y) frame.
 *  - Outside the image the label is OUTSIDE, larger than every pixel label.
 *    Triangles outside the image carry label 0xFFFF in the output (so a u16
 *    pixel label 0xFFFF cannot be told from the outside there).
 *  - Ownership: inputs stay owned by the caller and are only read; a host
 *    image may be reused once mesh_bitmap returns, a device image must stay
 *    valid until mesh_query reports the mesh done.  Outputs are device memory
 *    owned by the context, valid until mesh_release or mesh_destroy.
 *  - Threading: calls on one context are serialised by an internal mutex;
 *    work is ordered on the context's stream.
 */
#ifndef SBMT_H
#define SBMT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define SBMT_OK 0
#define SBMT_EINVAL (-1)    /* bad argument: dims, dtype, pitch, h, origin, mode */
#define SBMT_ENOMEM (-2)    /* device allocation failed */
#define SBMT_EPENDING (-3)  /* mesh_query poll: work not finished yet */
#define SBMT_ETIMEDOUT (-4) /* mesh_query: wait limit reached */
#define SBMT_ECAPACITY (-5) /* a cell holds more boundary vertices than the per-cell limit (mesh_stage 4 lists them) */
#define SBMT_EPROTO (-6)    /* requested mode is not available (SBMT_PREPROCESS in mesh_bitmap) */
#define SBMT_ECUDA (-7)     /* a CUDA call failed (message in sbmt_last_error) */
#define SBMT_EINTERNAL (-8) /* a device-side consistency check failed */
#define SBMT_ENOENT (-9)    /* unknown mesh handle or request */
#define SBMT_ECANCELED (-10) /* serving: the request was cancelled */

typedef struct sbmt_ctx sbmt_ctx;
typedef uint64_t sbmt_mesh;

enum { SBMT_U8 = 1, SBMT_U16 = 2, SBMT_F32 = 4 }; /* SBMT_F32: fields for mesh_project only */
enum { SBMT_PLAIN = 0, SBMT_PREPROCESS = 1 };
enum { SBMT_EXPLICIT = 0, SBMT_COMPACT = 1 };
/* sbmt_params.flags: SBMT_KEEP_STAGES keeps intermediate arrays for
 * mesh_stage; SBMT_DEBUG_STALL_SCAN is a test of the bound on device waits:
 * one tile of the counting scan withholds its sums, so that the wait of the
 * tile after it runs out (about one second) and the call returns
 * SBMT_ETIMEDOUT, leaving the context usable (for an image with at least
 * 4096 boundary segments; set on the first image of a batch). */
enum { SBMT_KEEP_STAGES = 1, SBMT_DEBUG_STALL_SCAN = 2 };

/* A label image.  width, height in 1..32768; pitch_bytes >= width * dtype
 * bytes; data is a host pointer (on_device = 0) or a device pointer of the
 * context's device (on_device = 1).  A device u16 image needs an even pitch
 * and an even address (SBMT_EINVAL otherwise). */
typedef struct {
  int32_t width, height;
  int64_t pitch_bytes;
  int32_t dtype; /* SBMT_U8 or SBMT_U16 */
  const void* data;
  int32_t on_device;
} sbmt_image;

/* Meshing parameters.  h = h_num / h_den pixels (Sec. 3.3's edge length);
 * the grid origin is (origin2x / 2, origin2y / 2).  h_num is even in
 * 2..1024 and h_den odd in 1..63 (else SBMT_EINVAL).  With origin2x and
 * origin2y even (the degeneracy-free class) no grid vertex lies on a pixel
 * line and no pixel corner on a grid edge, so every Alg. 1 event is a proper
 * crossing: the lattice path.  An odd one puts the origin on a pixel line
 * (a degenerate origin, e.g. (-1/2, -1/2) with origin2x = origin2y = -1):
 * grid vertices then lie on pixel lines and grid edges on the image
 * border, and mesh_bitmap meshes it by the general path -- the unmoved base
 * mesh, then the per-cell retriangulation of mesh_retriangulate, which takes
 * Alg. 1's vertex-on-segment and overlap incidences (explicit format; the
 * mesh numbered and coded as mesh_retriangulate's).  mesh_batch and
 * mesh_preprocess take even origins only.  mode is
 * SBMT_PLAIN or SBMT_PREPROCESS for mesh_bitmap (Alg. 3 in full, explicit
 * format only: see mesh_bitmap), SBMT_PLAIN for mesh_batch (SBMT_PREPROCESS
 * returns SBMT_EPROTO there) and SBMT_PREPROCESS for mesh_preprocess, which
 * reads the thresholds a, b, c.  format selects the storage
 * of the mesh (see sbmt_mesh_view): SBMT_EXPLICIT lists every triangle;
 * SBMT_COMPACT keeps the untouched base mesh implicit -- the paper's
 * "preserve the base mesh" (Sec. 1, Sec. 3.3) as a storage format. */
typedef struct {
  int32_t h_num, h_den;
  int32_t origin2x, origin2y;
  int32_t mode;
  double a, b, c;
  int32_t format;
  int32_t flags;
} sbmt_params;

/* A finished mesh (device pointers, owned by the context).
 *  xy    2 * n_vertices doubles: lattice vertices (row-major), then the
 *        boundary/grid-edge intersection vertices ordered by grid-edge id and
 *        position along the edge, then the boundary vertices inside cells
 *        ordered by cell id and pixel-corner id;
 *  tri   3 * n_triangles vertex ids, counter-clockwise, ordered by base cell
 *        id and then by the patch's emission order;
 *  label per triangle: label of the pixel holding its centroid, 0xFFFF outside;
 *  code  per triangle: bits 0-3 Alg. 1 bitmask of its cell (AB=2, BC=4,
 *        CA=8; bit 0 = a boundary vertex inside the cell), bits 4-5 the
 *        rotation sigma, bits 6-11 the key id (0 uncut, 1..15 table keys,
 *        63 outside Lemma 3.1's regime), bits 12-15 the (m,n) class as its
 *        1-based position in Thm. 3.2's list (0 = not applicable). */
typedef struct {
  int64_t n_vertices, n_triangles, n_cells, n_cut_cells, n_tierG_cells;
  int64_t n_segments;        /* boundary segments (maximal runs) */
  int64_t n_events;          /* boundary/grid-edge crossing vertices */
  int64_t n_inside_vertices; /* boundary vertices inside cells */
  int64_t n_lattice_vertices;
  int64_t n_tierG_triangles; /* triangles of cells outside the table's regime */
  const double* xy;
  const int32_t* tri;
  const uint16_t* label;
  const uint16_t* code;
  int32_t status; /* SBMT_OK, or the error the device work reported */
  /* SBMT_COMPACT meshes (format = SBMT_COMPACT; NULL / 0 otherwise):
   *  xy         2 * (n_vertices - n_lattice_vertices) doubles: the vertices
   *             after the lattice (ids n_lattice_vertices and up); lattice
   *             vertex coordinates are v(i, j) = o + h (i + j/2, sqrt3/2 j);
   *  cell_label per base cell: label of its triangle (A, B, C) when the cell
   *             is uncut (cell_code 0), 0xFFFF when cut;
   *  cell_code  per base cell: its pattern code (0 = uncut);
   *  patch_cell the cut cell ids, increasing (n_cut_cells of them);
   *  patch_off  n_cut_cells + 1 offsets: cut cell k's triangles are patch
   *             triangles patch_off[k] .. patch_off[k + 1] - 1;
   *  tri, label, code  the n_patch_triangles patch triangles, in cut-cell
   *             order, as in the explicit format.
   * Expanding them cell by cell (uncut cells emit (A, B, C)) gives the
   * explicit mesh exactly. */
  int32_t format;
  int64_t n_patch_triangles;
  const uint16_t* cell_label;
  const uint16_t* cell_code;
  const uint32_t* patch_cell;
  const uint32_t* patch_off;
} sbmt_mesh_view;

/* Create a context on CUDA device `device`.  pool_bytes (0 = no limit) is
 * the amount of freed device memory the context keeps cached for reuse;
 * cuda_stream is a cudaStream_t to order work on, or NULL for a stream the
 * context creates and owns. */
int mesh_create(sbmt_ctx** ctx, int device, size_t pool_bytes, void* cuda_stream);

/* Mesh one image (Sec. 3.3 grid, Alg. 1 classification, Alg. 2 lookup).
 * Enqueues the work on the context's stream and returns a handle; the call
 * synchronises with the device once, after counting the image's boundary
 * segments and their grid crossings, to size its buffers.  The mesh is
 * complete when mesh_query returns SBMT_OK.  SBMT_ETIMEDOUT: a bounded
 * device wait ran out (see SBMT_DEBUG_STALL_SCAN).
 * With params->mode = SBMT_PREPROCESS (and the explicit format) the call
 * runs Alg. 3 in full, in the pipelined schedule of Sec. 3.5's corollary:
 * Regions I-II (mesh_preprocess), then Region III, Alg. 2 on the
 * preprocessed mesh T (mesh_retriangulate); the returned mesh is the
 * embedded one, and T is released.  That path synchronises three times. */
int mesh_bitmap(sbmt_ctx* ctx, const sbmt_image* img, const sbmt_params* params, sbmt_mesh* out);

/* Region III of Alg. 3's schedule: Alg. 2, the template retriangulation,
 * applied to the explicit counter-clockwise mesh `base` (normally one made by
 * mesh_preprocess; any mesh whose cells are counter-clockwise and whose edges
 * have at most two cells) against the boundary of img, each cell on its own
 * from its local intersection class (Sec. 3.5, corollary on lookup-driven
 * parallel retriangulation).  base stays valid; out receives a new mesh:
 *  xy    base's vertices in their ids, then the boundary events on base's
 *        edges ordered by owning cell (the smaller of the two cells beside
 *        the edge), its local edge and the position from the edge's lower-id
 *        end, then the boundary vertices inside cells by cell and
 *        pixel-corner id;
 *  tri   by base cell, then the patch order;
 *  label the pixel holding ((x1 + x2) + x3) / 3, 0xFFFF outside;
 *  code  as for mesh_bitmap: Alg. 1's bitmask (an event sets its edge, a
 *        base vertex on a boundary piece -- a vertex on the segment -- both
 *        edges at it, an edge lying on a boundary run -- an overlap -- its
 *        own bit, bit 0 a boundary vertex inside), the rotation, the key (1..15
 *        table keys, 63 greedy), the (m, n) class; 0 for cells left as they
 *        are.
 * An event of a base edge is a point of the open edge where the boundary
 * meets it: a crossing of a boundary pixel edge, or a pixel corner on the
 * edge with a boundary pixel edge not collinear with it; on the horizontal
 * pixel line y0 it is x = P.x + ((y0 - P.y) (Q.x - P.x)) / (Q.y - P.y) with
 * P the edge's lower-id end (vertical lines likewise), every operation
 * rounded once in double precision.  Cells in the table's regime (no piece
 * ending at a corner of the cell, every event ending one piece, no inside
 * vertex and one or two chords, or one inside vertex every piece ends at)
 * take the App. G template of their key; the others the greedy rule (vertex
 * pairs by squared length rounded to single precision, ties by local index
 * pair, kept when the open segment holds no vertex and crosses no kept
 * edge).  Per-cell limits: 16 events on an edge, 16 inside vertices, 48
 * nodes (SBMT_ECAPACITY past them).  mesh_query reports n_cut_cells,
 * n_tierG_cells and _triangles, n_events, n_inside_vertices and, as
 * n_lattice_vertices, base's vertex count.  Synchronises once. */
int mesh_retriangulate(sbmt_ctx* ctx, const sbmt_image* img, sbmt_mesh base, sbmt_mesh* out);

/* A mesh of the caller's own as an explicit mesh handle, e.g. the base mesh
 * of mesh_retriangulate (Alg. 2 applies to any conforming counter-clockwise
 * triangulation, Sec. 3.5).  xy: 2 * n_vertices doubles (x, y in pixel
 * coordinates, pixel (i, j) covering [i - 1/2, i + 1/2] x [j - 1/2, j + 1/2]),
 * tri: 3 * n_triangles vertex ids; both HOST arrays, copied before the call
 * returns (the caller keeps ownership).  The handle's labels are 0xFFFF and
 * its codes 0; mesh_query reports n_cells = n_triangles and
 * n_lattice_vertices = n_vertices, its other counts 0.  SBMT_EINVAL
 * (checked on the host before ctx is used): a null array, fewer than 3
 * vertices or 1 triangle, 2^31 or more vertices or triangle ids, a
 * coordinate that is not finite or beyond 2^24 px, an id outside
 * [0, n_vertices) or repeated in a triangle.  Orientation and edge
 * manifoldness are mesh_retriangulate's checks (SBMT_EINTERNAL).
 * Synchronises once. */
int mesh_import(sbmt_ctx* ctx, const double* xy, int64_t n_vertices, const int32_t* tri, int64_t n_triangles,
                sbmt_mesh* out);

/* Geometric preprocessing of the base mesh (Alg. 3, Steps 1-3): the mesh T
 * that Alg. 3's template retriangulation starts from.  params->mode must be
 * SBMT_PREPROCESS and params->format SBMT_EXPLICIT.  The thresholds a, b, c
 * are relative to the reference edge length sqrt(0.45) px of the paper's
 * experiments (Sec. 4, App. I: a = 0.26, b = 0.125, c = 0.183 is
 * admissible), so in pixels they are a h / sqrt(0.45) etc.; they must lie
 * in the admissible range b < a/2, c < a/sqrt2 (Eq. "admissible range") and
 * a < h/2, else SBMT_EINVAL.  Boundary points are the PSLG vertices, the
 * pixel corners with id y (W + 1) + x; boundary segments are the boundary
 * pixel edges.
 *  Step 1  a lattice vertex moves onto the boundary point nearest to it when
 *          that point is closer than a (ties: the smaller id);
 *  Step 2  a vertex that did not snap moves away from the nearest point q of
 *          the boundary segments (ties: the smaller pixel-edge id, horizontal
 *          edge (m, k) between pixels (m, k-1) and (m, k) has id k W + m,
 *          vertical edge (m, k) between (m-1, k) and (m, k) has id
 *          (H + 1) W + k (W + 1) + m) along q -> v to distance c, when q is
 *          closer than c;
 *  Step 3  a boundary point p closer than b to an edge e of the moved mesh,
 *          neither end of e at p, is a candidate (p, e).  It applies when e
 *          is p's smallest candidate edge (by smaller end id, then larger)
 *          and no smaller point is a candidate on an edge of the triangles
 *          beside e, and when the halves below all stay strictly
 *          counter-clockwise.  p becomes vertex n_lattice_vertices + (its
 *          rank by id among the applied points), and each triangle
 *          (u, w, x) beside e = u w becomes (u, p, x) and (p, w, x).
 * Steps 1 and 2 read the lattice positions; a vertex of the base mesh's
 * outer boundary snaps only onto an image corner or a border point at least
 * h + a from both ends of its side (so that T covers the image); every
 * distance test is a
 * double-precision comparison of squared distances.  The result is an
 * explicit mesh (mesh_query): the lattice vertices in id order (moved),
 * then the inserted points; the cells in id order, a split cell's two
 * halves in place of it; labels from the centroids as for mesh_bitmap;
 * code 0 everywhere; n_cut_cells counts the split cells.  mesh_quality and
 * mesh_project accept it.  Synchronises with the device once. */
int mesh_preprocess(sbmt_ctx* ctx, const sbmt_image* img, const sbmt_params* params, sbmt_mesh* out);

/* Records of a preprocessed mesh (waits for it):
 *  status  per lattice vertex (device, n_lattice_vertices bytes): 0 kept,
 *          1 snapped (Step 1), 2 repelled (Step 2);
 *  snap    per lattice vertex (device, int32): the corner id snapped to, -1;
 *  elim    per applied Step 3 candidate, by point id (device, 3 int32):
 *          the point's corner id and the removed edge's ends u < w;
 *  n_points the boundary points; n_candidate_points those with a candidate;
 *  a_px, b_px, c_px the thresholds in pixels.
 * SBMT_EINVAL for a mesh not made by mesh_preprocess. */
typedef struct {
  int64_t n_lattice_vertices, n_points;
  int64_t n_snapped, n_repelled, n_candidate_points, n_eliminated, n_split_cells;
  double a_px, b_px, c_px;
  const uint8_t* status;
  const int32_t* snap;
  const int32_t* elim;
} sbmt_pre_info;
int mesh_preprocess_info(sbmt_ctx* ctx, sbmt_mesh mesh, sbmt_pre_info* out);

/* Mesh n images of any sizes together (the batched form of the data-parallel
 * path, Sec. 3.5's corollary: every cell's patch is independent); params
 * points to n parameter sets, or to one shared by all (n_params = 1).  out
 * receives n handles.  Every stage runs as one launch over all n images:
 * a counting phase, one host synchronisation for the whole batch, and an
 * emission phase whose variable-size stages (cut cells, Tier-G cells, the
 * registry's large buckets) are persistent kernels over batch-wide work
 * queues, the Tier-G cells of all images ordered by size.  The emission
 * phase runs as a CUDA graph when the tuning of the batch's size class says
 * so (mesh_autotune).  Each mesh is identical to the one mesh_bitmap makes
 * for its image.  A failing image fails the whole batch (no handles).  The
 * meshes of a batch share one device block, freed with the last of them. */
int mesh_batch(sbmt_ctx* ctx, const sbmt_image* imgs, int n, const sbmt_params* params, int n_params,
               sbmt_mesh* out);

/* Tune the batched path for the size class of this batch (image count and
 * total pixels, each log2, and the largest h, log2 rounded): mesh the batch
 * repeatedly (1 + repeats runs per candidate, meshes released) under
 * candidate launch parameters -- persistent blocks per SM of the cut-cell
 * kernel (4..16) and of the Tier-G kernel (8..32), Tier-G on side streams or
 * not, the emission phase as a CUDA graph or not -- by coordinate descent
 * from the defaults, and keep the fastest for the class, in the context and
 * appended to the tuning file (environment SBMT_TUNE_FILE, else
 * $HOME/.cache/sbmt_tune.txt) that every context reads on its first batch.
 * No counterpart in the paper (which has no parallel implementation). */
int mesh_autotune(sbmt_ctx* ctx, const sbmt_image* imgs, int n, const sbmt_params* params, int n_params,
                  int repeats);
/* The launch parameters mesh_batch would use for this batch: cut-cell
 * blocks per SM, Tier-G blocks per SM, fork (0/1), graph (0/1). */
int mesh_tuning(sbmt_ctx* ctx, const sbmt_image* imgs, int n, const sbmt_params* params, int n_params,
                int32_t* out4);
/* Set, for this context only, the launch parameters of this batch's size
 * class (the four values of mesh_tuning; SBMT_EINVAL outside cut-cell
 * blocks 1..16, Tier-G blocks 1..32, fork and graph 0/1). */
int mesh_set_tuning(sbmt_ctx* ctx, const sbmt_image* imgs, int n, const sbmt_params* params, int n_params,
                    const int32_t* in4);

/* Check an image and its parameters as mesh_bitmap does, with no device
 * work: SBMT_OK, SBMT_EINVAL or SBMT_EPROTO. */
int mesh_check(const sbmt_image* img, const sbmt_params* params);

/* The device bytes a mesh holds until it is released (its outputs, and its
 * kept stages with SBMT_KEEP_STAGES); known as soon as mesh_bitmap or
 * mesh_batch returns. */
int mesh_footprint(sbmt_ctx* ctx, sbmt_mesh mesh, size_t* bytes);

/* Wait up to wait_ms milliseconds (0 = poll, < 0 = no limit) for a mesh and
 * fill *out.  Returns SBMT_EPENDING / SBMT_ETIMEDOUT while unfinished, or
 * the mesh's status. */
int mesh_query(sbmt_ctx* ctx, sbmt_mesh mesh, int wait_ms, sbmt_mesh_view* out);

/* Free the device memory of one mesh (waits for its work first). */
int mesh_release(sbmt_ctx* ctx, sbmt_mesh mesh);

/* Release every mesh and destroy the context. */
int mesh_destroy(sbmt_ctx* ctx);

/* Intermediate arrays of a finished mesh made with SBMT_KEEP_STAGES, copied
 * to host memory, for checking each step on its own (stage 4 is kept for
 * every mesh):
 *  stage 1 boundary segments, 8 int32 each: corner x, corner y, direction
 *          (0 +x, 1 +y), length, label below/left, label above/right (0xFFFF
 *          = outside), reversed (1 when the lower label lies left of -x/-y),
 *          0;
 *  stage 2 grid-edge events in vertex-id order, 4 int64 each: grid-edge id,
 *          vertex id, packed segment start corner (y * (W + 1) + x), dir;
 *  stage 3 cut cells in id order, 5 int64 each: cell id, code, triangles,
 *          boundary vertices inside, outside-regime flag;
 *  stage 4 the cells whose local boundary graph has more vertices than the
 *          per-cell limit of the Tier-G rule (64), the reason for the status
 *          SBMT_ECAPACITY: their ids in increasing order, 1 int64 each, the
 *          first 1024 of them; *n is their total number (0 for a mesh made
 *          by mesh_preprocess, which has no stages 1-3).
 * Writes min(n, cap) records to host_out and the total count to *n. */
int mesh_stage(sbmt_ctx* ctx, sbmt_mesh mesh, int stage, void* host_out, int64_t cap, int64_t* n);

/* Quality measures of a finished mesh, computed on the device from its
 * output (the measures of the paper's experiments, Sec. 4: Tables "mesh
 * quality", "comparison", "aspect-ratio statistics", Fig. "minimum angle
 * histograms").  Angles, areas and aspect ratios in double precision from
 * the output coordinates, in pixel units:
 *  min_angle_deg  smallest interior angle over all triangles;
 *  min_area       smallest triangle area;
 *  slivers        triangles whose smallest angle is below 5 degrees;
 *  equilateral    triangles whose longest and shortest squared edges differ
 *                 by at most 1e-9 of the longest (the edge-length test);
 *  area_mean, area_var  mean and population variance of the areas;
 *  ar_median, ar_p95, ar_max  AR = longest edge / shortest altitude; the
 *                 percentiles are nearest-rank (the ceil(p T)-th smallest)
 *                 of AR rounded to single precision, the maximum in double;
 *  angle_hist     smallest angles in 2-degree bins [0,2) ... [58,60].
 * Needs a mesh in the SBMT_EXPLICIT format (SBMT_EINVAL otherwise).
 * Waits for the mesh; synchronises with the device a few times. */
typedef struct {
  int64_t triangles;
  double min_angle_deg, min_area;
  int64_t slivers, equilateral;
  double area_mean, area_var;
  double ar_median, ar_p95, ar_max;
  int64_t angle_hist[30];
} sbmt_quality;
int mesh_quality(sbmt_ctx* ctx, sbmt_mesh mesh, sbmt_quality* out);

/* Projection of a scalar pixel field onto a finished mesh (Sec. 3.3: the
 * bitmap's scalar fields are projected onto each triangle; Sec. 3.6 and
 * App. C: the interpolation stage, constant work per triangle).
 *  field         a width x height image of the meshed size with dtype
 *                SBMT_F32 (4-byte floats), host or device (see sbmt_image;
 *                a host field is copied first);
 *  tri_value     device, n_triangles floats, or NULL: per triangle T the
 *                mean of the piecewise-constant pixel field over T,
 *                (1/|T|) sum_p f_p |T n p|, pixel (x, y) the unit square
 *                centred at (x, y); 0 for triangles outside the image;
 *  vertex_value  device, n_vertices floats, or NULL: the bilinear
 *                interpolation of the field between pixel centres at each
 *                vertex, the point clamped to [0, W-1] x [0, H-1].
 * Single precision, double for thin triangles (longest edge L with
 * L (L + 1) > 64 |T|): a triangle's mean is within a few 2^-24
 * L (L + 1) / |T| of the field's range over its pixels.  Both buffers are
 * caller-owned.  The work is enqueued on the context's stream after the
 * mesh; mesh_query on the mesh then also waits for it.  Explicit meshes
 * only: SBMT_EINVAL for a compact mesh, a field of another size or dtype,
 * or a mesh of 2^32 triangles or more. */
int mesh_project(sbmt_ctx* ctx, sbmt_mesh mesh, const sbmt_image* field, float* tri_value, float* vertex_value);

/* Transient heat diffusion on a label region of a finished mesh (App. H:
 * du/dt = alpha Lap u on the region, u = 0 on its boundary, from a centred
 * Gaussian pulse).  The region is the set of triangles of label `label`; its
 * boundary vertices (those also on a triangle of another label, 0xFFFF
 * outside the image included) stay at 0, and the other vertices of the
 * region are free.  Linear finite elements (the paper names no scheme):
 *  - K, the cotangent stiffness: a triangle with angle theta_k at corner k
 *    adds -cot(theta_k)/2 to K_ij and K_ji for the opposite edge ij and
 *    cot(theta_k)/2 to K_ii and K_jj;
 *  - M, the lumped mass: a third of the area of each region triangle at a
 *    vertex;
 *  - backward Euler: (M + alpha dt K) u_{n+1} = M u_n on the free vertices.
 * Each step is solved by conjugate gradients with the diagonal as
 * preconditioner, started from u_n, until |r| <= tol |b|, in double
 * precision.
 *  u0 = amplitude exp(-|x - (x0, y0)|^2 / (2 sigma^2)) at the free vertices
 *  (pixel units; alpha in px^2 per unit time).
 *  u           device, n_vertices doubles: u after `steps` steps (0 outside
 *              the region and on its boundary);
 *  peaks       host, `steps` doubles, or NULL: the maximum of u after each
 *              step;
 *  iterations  host, `steps` int32, or NULL: the CG iterations of each step.
 * Explicit meshes only (SBMT_EINVAL otherwise, or for bad parameters).
 * SBMT_ETIMEDOUT if a step does not converge within max_iterations.  Runs on
 * the context's stream after the mesh and returns when done. */
typedef struct {
  int32_t label;
  double alpha, dt;
  int32_t steps;
  double x0, y0, sigma, amplitude;
  double tol;
  int32_t max_iterations;
} sbmt_heat_params;
int mesh_heat(sbmt_ctx* ctx, sbmt_mesh mesh, const sbmt_heat_params* params, double* u, double* peaks,
              int32_t* iterations);

/* Per-kernel device time, for tracing and roofline accounting (no
 * counterpart in the paper, which reports no timings).  With enable != 0
 * every kernel launch of the context is bracketed by two CUDA events on the
 * context's stream.  mesh_profile_read waits for the recorded events and
 * writes, for each of the *n kernels of the hot path (at most cap), its
 * name (static string), accumulated milliseconds and launch count; reset
 * != 0 clears the totals. */
int mesh_profile(sbmt_ctx* ctx, int enable);
int mesh_profile_read(sbmt_ctx* ctx, int reset, int cap, const char** names, double* ms, int64_t* launches,
                      int* n);

/* Boundary extraction without any device allocation (no counterpart in the
 * paper: an interface for callers that may not allocate device memory, such
 * as a host application that gives the library a fixed device budget, or a
 * latency-critical path where an allocation could block or fail).
 *
 * Extracts the boundary segments of one device-resident image -- the first
 * step of mesh_bitmap -- on the calling thread's current CUDA device and
 * enqueues the work on cuda_stream (NULL = the legacy default stream).
 *  d_image     device image, width x height in 1..4096 (larger images return
 *              SBMT_EINVAL), pitch_bytes >= width * dtype, dtype SBMT_U8 or
 *              SBMT_U16;
 *  d_segments  device output, room for `capacity` records of 4 int32 each:
 *              corner x, corner y, length | direction << 30 (0 +x, 1 +y) |
 *              reversed << 31, label below/left | label above/right << 16
 *              (0xFFFF outside the image); records come in no fixed order;
 *  d_count     device u32 receiving the number of segments (it may exceed
 *              capacity, then only `capacity` records are written), or
 *              0xFFFFFFFF when the extraction met an inconsistency (a run
 *              with no end vertex; never for a valid image).
 * A u16 image needs an even pitch and an even address (SBMT_EINVAL
 * otherwise).  Launch errors are read with cudaGetLastError, which also
 * returns, and clears, an error still pending from the caller's earlier
 * work on this thread.
 * Working memory is one 8 MiB array of static device storage held by every
 * GPU that loads the library until the process exits; the call allocates
 * and frees nothing.  The first call on a device looks up the array's device
 * address (make it before any stream capture).  Every call shares the
 * array, so calls whose work overlaps on the GPU race: order them on one
 * stream or synchronise between them.  Returns SBMT_OK once the work is
 * enqueued; the message of a failing call is in sbmt_static_last_error(). */
int sbmt_extract_segments_static(const void* d_image, int32_t width, int32_t height, int64_t pitch_bytes,
                                 int32_t dtype, void* d_segments, uint32_t capacity, uint32_t* d_count,
                                 void* cuda_stream);
const char* sbmt_static_last_error(void);

/* ------------------------------------------------------------------------
 * Serving: a request loop for meshing requests of different sizes (no
 * counterpart in the paper, whose prototype meshes one image at a time; the
 * independence of every cell's patch, Sec. 3.5's corollary, is what makes a
 * request's mesh the same alone and among others).
 *
 * server_submit queues a request and returns at once.  Requests are admitted
 * in arrival order by device memory: before its boundary is counted a
 * request reserves an upper bound of the device bytes meshing it can hold,
 * computed from its width, height and h alone (every pixel edge a boundary
 * edge crossing as many grid edges as its length allows); once its batch's
 * counting phase is done the reservation becomes the exact size of its mesh
 * (mesh_footprint), held until server_release.  A request is admitted when
 * the reservations stay within the budget and its bound fits the device's
 * free memory; one whose bound exceeds the budget fails with SBMT_ENOMEM.
 * Admitted requests are meshed in batches (mesh_batch: every stage one
 * launch over the batch).  Continuous batching: each worker (a context with
 * its own stream and host thread) takes the next batch as soon as its
 * previous batch's counting phase is done, so requests that arrive while
 * others are on the GPU join the next launch, and the workers' batches
 * overlap on the device.  Bitmaps passed as device pointers (which must stay
 * valid until the request is done) and every finished mesh stay on the
 * device.  A request's mesh is identical to mesh_bitmap's for its image,
 * whatever it was batched with.
 * ------------------------------------------------------------------------ */
typedef struct sbmt_server sbmt_server;
typedef struct {
  size_t hbm_budget;  /* device bytes reservations may hold; 0 = 90% of the free memory at creation */
  int32_t max_batch;  /* requests per batch (0 = 64) */
  int32_t workers;    /* contexts taking batches in turn (0 = 2) */
  int32_t oom_every;  /* fault injection on the host: every k-th admission check sees no free memory (0 = off) */
} sbmt_server_config;
typedef struct {
  int32_t status;     /* SBMT_OK, or the request's error (SBMT_ECANCELED, SBMT_ENOMEM, ...) */
  int32_t batch_size; /* requests meshed in the same batch */
  double queued_ms;   /* submit to admission into a batch */
  double total_ms;    /* submit to the mesh found finished by the server */
} sbmt_request_info;
typedef struct {
  int64_t submitted, completed, failed, cancelled, batches, queued;
  int64_t reserved_bytes, peak_reserved_bytes, budget_bytes;
} sbmt_server_stats;

/* The reservation of a request before its boundary is counted: an upper
 * bound of the device bytes meshing this image can hold (its outputs and
 * the path's working memory), from its width, height, dtype and h alone --
 * every pixel edge a boundary edge, every corner a boundary vertex, and
 * every boundary edge crossing as many grid edges as its length allows (a
 * unit pixel edge meets at most 3 + 2.31/h of them). */
int mesh_bound(const sbmt_image* img, const sbmt_params* params, size_t* bytes);
/* Start a server on a device (cfg may be NULL for the defaults). */
int server_create(sbmt_server** srv, int device, const sbmt_server_config* cfg);
/* Queue a request (checked as by mesh_check first: SBMT_EINVAL or
 * SBMT_EPROTO and no request for a malformed one).  A host image is copied
 * before the call returns. */
int server_submit(sbmt_server* srv, const sbmt_image* img, const sbmt_params* params, uint64_t* request);
/* Wait up to wait_ms milliseconds (0 = poll, < 0 = no limit) for a request:
 * SBMT_EPENDING / SBMT_ETIMEDOUT while unfinished, else its status; view
 * (device pointers, valid until server_release) and info may be NULL. */
int server_wait(sbmt_server* srv, uint64_t request, int wait_ms, sbmt_mesh_view* view, sbmt_request_info* info);
/* Cancel a request: a queued one finishes at once with SBMT_ECANCELED; a
 * running one is released (and forgotten) when its batch is done. */
int server_cancel(sbmt_server* srv, uint64_t request);
/* Free a finished request's mesh and forget the request. */
int server_release(sbmt_server* srv, uint64_t request);
int server_stats(sbmt_server* srv, sbmt_server_stats* out);
/* Stop the server: queued requests are dropped, running ones finished, and
 * every mesh freed. */
int server_destroy(sbmt_server* srv);
const char* sbmt_server_last_error(void);

/* Message of the last failing call on this thread (never NULL). */
const char* sbmt_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SBMT_H */
