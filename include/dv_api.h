/*
 * dv_api.h — C ABI of the B300 (sm_103a) differentiable-voxelization library.
 *
 * The library evaluates the generalized winding number of a triangle mesh,
 *
 *     w(q) = (1/4pi) * sum_f Omega_f(q),                       Eq. (5), Algorithm 1
 *     Omega_f(q) = 2 * ATAN2(det(a,b,c), D),                   Eq. (7) with Eq. (8)
 *     a = v0 - q, b = v1 - q, c = v2 - q,
 *     D = |a||b||c| + (a.b)|c| + (b.c)|a| + (c.a)|b|,
 *
 * for every query point against every face (no hierarchy, §1), the
 * binarised occupancy w > 0.5 (§2.1, Eq. (3); the threshold is this
 * library's reading, the paper states none), and the adjoint
 * dL/dV = sum_q (dL/dw_q) dw_q/dV that makes the voxelization
 * differentiable (§1 contributions, §2.4).
 *
 * Conventions shared by every entry point:
 *   - Buffers marked d_ are DEVICE pointers on the current CUDA device; the
 *     caller owns and allocates them (for example through PyTorch). h_ marks
 *     a host pointer. Nothing here takes ownership of a caller buffer.
 *   - Vertices: float32 [nv][3], row-major. Faces: int32 [nf][3], indices into
 *     the vertex array, counter-clockwise seen from outside (then w = +1 inside).
 *   - Grids are cell-centred: x_i = lo + (i + 1/2)(hi - lo)/n per axis, and the
 *     linear query index is (iz * ny + iy) * nx + ix (x fastest).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Every call is stream-ordered and returns without waiting for the GPU,
 *     unless its comment says it synchronizes.
 *   - Host-detectable errors (bad arguments, bad sizes) are returned
 *     synchronously and nothing is enqueued. Launch errors are reported as
 *     DV_ERR_CUDA. dv_last_error() gives a thread-local detail string.
 *   - There is no CPU fallback: a call either runs on the GPU or fails.
 *   - A dv_mesh owns device memory from the stream-ordered allocator (cudaMallocAsync
 *     on the calling stream); scratch grows on first use unless reserved.
 *   - A dv_mesh owns scratch memory. Forward calls (dv_winding, dv_voxelize_grid)
 *     on the same mesh must be ordered with each other (one stream, or events),
 *     and so must backward calls; a forward and a backward on the same mesh use
 *     separate scratch and may run concurrently on two streams once the mesh
 *     is packed and its scratch reserved (dv_mesh_reserve). Different meshes are
 *     independent. Calls on one mesh come from one host thread at a time (the
 *     mesh's host state, such as grown scratch or the boundary edges built on
 *     first use, is not locked).
 */
#ifndef DV_API_H
#define DV_API_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DV_ABI_VERSION 1

typedef enum {
    DV_OK = 0,
    DV_ERR_INVALID_ARG = 1,   /* null pointer, negative size, bad grid, bad enum */
    DV_ERR_INVALID_MESH = 2,  /* face index outside [0, nv) or non-finite vertex */
    DV_ERR_OOM = 3,           /* device allocation for mesh storage/scratch failed */
    DV_ERR_CUDA = 4,          /* a CUDA call or kernel launch failed */
    DV_ERR_TIMEOUT = 5,       /* a bounded device-side wait ran out (see dv_mesh_check) */
    DV_ERR_UNSUPPORTED = 6    /* valid request this build does not handle (e.g. size limits) */
} dv_status;

/* Arithmetic of the forward pass.
 *   DV_PREC_FP32        FP32 per-pair terms, plain FP32 sum over faces.
 *   DV_PREC_FP32_KAHAN  FP32 per-pair terms, compensated (Kahan) sum over blocks of faces.
 *   DV_PREC_MIXED       DV_PREC_FP32_KAHAN, then every query with |w - 0.5| < 1e-3 or
 *                       within 1e-3 (Euclidean) of a triangle is re-evaluated over all
 *                       faces in FP64 on the GPU and its w / occupancy overwritten.
 *   DV_PREC_FP16        ablation of the paper's half precision (§3.1): per-pair terms in
 *                       packed FP16 arithmetic (offsets and their partial sums in FP32),
 *                       FP32 Kahan sums; grid queries only; NOT accurate to 1e-4.
 * The paper ran half precision (§3.1); the other modes are this library's choice. */
typedef enum { DV_PREC_FP32 = 0, DV_PREC_FP32_KAHAN = 1, DV_PREC_MIXED = 2, DV_PREC_FP16 = 3 } dv_precision;

/* Cell-centred voxel grid over the box [lo, hi] (§3: meshes normalized to [-1,1],
 * resolutions 32..256; any n >= 1 per axis is accepted). */
typedef struct {
    float lo[3];
    float hi[3];
    int32_t n[3];
} dv_grid;

/* Opaque handle: packed per-face records resident on the device, the
 * vertex-to-face adjacency used by the backward scatter, and scratch. */
typedef struct dv_mesh dv_mesh;

/* Filled by dv_voxelize_grid when a report is requested (that call then synchronizes). */
typedef struct {
    int64_t n_queries;           /* queries evaluated */
    int64_t n_faces;             /* faces per query */
    int64_t n_flagged;           /* queries selected for FP64 re-evaluation (DV_PREC_MIXED) */
    int64_t n_occ_changed;       /* of those, how many changed occupancy after FP64 */
    double max_abs_fp32_vs_fp64; /* max |w_fp32 - w_fp64| over the re-evaluated queries */
} dv_report;

/* Version of this ABI (DV_ABI_VERSION). */
int dv_abi_version(void);

/* Report of the bounds checks of the debug build (no counterpart in the paper).
 * The debug build of this library (libdv_debug.so, the same sources compiled
 * with -DDV_DEBUG) checks the index of every indexed global access of the hot
 * kernels against its buffer's length; an index outside it is counted, the
 * first is recorded, and the access is skipped instead of faulting. Outputs
 * (host pointers, all required): *count = the number of rejected accesses
 * since the last clear; *site, *index, *bound = the first one's site code
 * (1 forward tile copy, 2 forward output, 3 flagged list, 4 split partials,
 * 5 FP64-pass event, 6 FP64-pass query, 7 adjoint record, 8 upstream, 9 face
 * gradient, 10 vertex gather, 11 near-surface flag, 12 packing), its index and
 * the length it was checked against. clear != 0 resets the records. Reads
 * device memory synchronously (waits for the device). The release build
 * returns DV_ERR_UNSUPPORTED. */
dv_status dv_debug_report(int64_t *count, int32_t *site, int64_t *index, int64_t *bound, int clear);

/* Self-test of the bounded waits used by every shared-memory copy pipeline of
 * this library (no counterpart in the paper). One CTA waits on a barrier phase
 * with a limit of limit_us microseconds (1 .. 1e7). With arrive != 0 the phase
 * completes and the call returns DV_OK; with arrive == 0 nothing arrives, the
 * wait gives up after the limit, the kernel records and returns
 * DV_ERR_TIMEOUT, and the CUDA context stays usable. Synchronizes `stream`. */
dv_status dv_selftest_bounded_wait(int64_t limit_us, int arrive, void *stream);

/* Self-test of the give-up path of the forward's shared-memory copy pipeline
 * (no counterpart in the paper). Runs the grid forward of dv_winding (strip
 * order, Kahan FP32) on `mesh` over `grid` into d_out_w (float32, caller-owned
 * device memory, nx*ny*nz values), except that in every CTA the copy of tile
 * `skip_tile` (an index into the CTA's own run of 96-event tiles, >= 0) is
 * never issued and every wait is limited to limit_us microseconds (1 .. 1e7).
 * A CTA that reaches that tile waits for the limit, stops issuing copies, waits
 * (bounded) for the copies it has in flight, records DV_ERR_TIMEOUT in the
 * mesh's sticky error word and finishes; its values in d_out_w are then not
 * meaningful. With skip_tile beyond every CTA's last tile the call is an
 * ordinary forward. Synchronizes `stream` and returns the error word without
 * clearing it (DV_ERR_TIMEOUT, or DV_OK); dv_mesh_check then reports it once.
 * No fault, trap or unbounded wait is involved. */
dv_status dv_selftest_forward_timeout(dv_mesh *mesh, const dv_grid *grid, float *d_out_w, int64_t skip_tile,
                                      int64_t limit_us, void *stream);

/* Strip order of a mesh's faces, the visiting order of the forward passes
 * (the sum of Eq. (5) is order-free; this order lets consecutive faces share
 * the per-vertex |v - q| and per-edge dot terms of Eq. (7)). HOST function, no
 * GPU needed. faces int32 [nf][3] (host), indices in [0, nv). Output, host,
 * caller-owned: events ev_vert[k] (a vertex index) and ev_face[k] (the face
 * completed by this event and the two events before it, or -1 for the first
 * two events of each strip). Every face appears exactly once; the vertex set
 * {ev_vert[k-2], ev_vert[k-1], ev_vert[k]} of an event with ev_face[k] >= 0
 * equals that face's vertex set. nf <= n_events <= 3 nf. With ev_vert or
 * ev_face NULL only *n_events is set (size query); DV_ERR_INVALID_ARG if
 * capacity < *n_events. No counterpart in the paper (an evaluation order of
 * this library). */
dv_status dv_build_strips(const int32_t *faces, int64_t nf, int64_t nv, int32_t *ev_vert, int32_t *ev_face,
                          int64_t capacity, int64_t *n_events);

/* Edge-sharing face pairs of the adjoint (grid and query lists): consecutive faces of the strip
 * order (dv_build_strips) taken two at a time, so that per (query, pair) four
 * vertex distances and five edge dots of the derivative of Eq. (7) serve two
 * faces. HOST function, no GPU needed. faces int32 [nf][3] (host), indices in
 * [0, nv). Output, host, caller-owned: pairs int32 [n_pairs][8] = p0, p1, p2,
 * p3, fA, fB, code, 0 with face fA = (p0, p1, p2) in its input orientation
 * (a rotation of its corners) and face fB the vertex set {p1, p2, p3}, taken
 * as (p2, p1, p3); code holds for each corner c = 0, 1, 2 of (p0, p1, p2) the
 * input corner of fA it is (bits 2c), for each corner of (p2, p1, p3) the
 * input corner of fB (bits 6 + 2c), and bit 12 when fB's input orientation is
 * the reverse of (p2, p1, p3); singles int32 [n_singles] = the faces in no
 * pair. Every face is in exactly one pair or in singles. With pairs or singles
 * NULL only the counts are set (size query); DV_ERR_INVALID_ARG if a capacity
 * is below its count. No counterpart in the paper (an evaluation order). */
dv_status dv_build_face_pairs(const int32_t *faces, int64_t nf, int64_t nv, int32_t *pairs, int32_t *singles,
                              int64_t capacity_pairs, int64_t capacity_singles, int64_t *n_pairs,
                              int64_t *n_singles);

/* Human-readable name of a status code. Never NULL. */
const char *dv_status_string(dv_status s);

/* Detail of the last error returned on the calling host thread ("" if none). */
const char *dv_last_error(void);

/* Algorithm 1 input "Mesh (V, F)": validate the faces (every index in [0, nv))
 * and vertices (finite), then pack each face f into a per-face record
 * (v0, v1, v2 and the face normal (v1-v0)x(v2-v0), FP32 and FP64 copies),
 * build the vertex-to-face adjacency, the strip order of the faces
 * (dv_build_strips) with its per-event records, used by the grid forward
 * and the FP64 re-evaluation, and the edge-sharing face pairs of the
 * adjoint (dv_build_face_pairs). The mesh keeps a host copy of the faces (for
 * the boundary edges, found on first use). d_verts float32 [nv][3], d_faces
 * int32 [nf][3] are read only during this call (the mesh keeps its own copies).
 * SYNCHRONIZES `stream` (for the validation result, and once the uploads are
 * done). nv >= 3, nf >= 1. On success *out receives a new handle; release it
 * with dv_mesh_destroy. */
dv_status dv_mesh_create(const float *d_verts, int64_t nv, const int32_t *d_faces, int64_t nf, void *stream,
                         dv_mesh **out);

/* Re-pack the face records from new vertex positions (same nv, same faces):
 * the morphing loop of §2.4 moves vertices every step. Stream-ordered, no sync,
 * no validation of finiteness. */
dv_status dv_mesh_update_verts(dv_mesh *mesh, const float *d_verts, void *stream);

/* Pre-size the mesh's scratch so that later forward/backward calls on `grid`
 * (may be NULL) or on query lists of up to max_list_queries points allocate
 * nothing (useful before timing or CUDA-graph capture). Without it, scratch
 * grows on first use. Allocates on the stream of the mesh's most recent call
 * and synchronizes that stream. */
dv_status dv_mesh_reserve(dv_mesh *mesh, const dv_grid *grid, int64_t max_list_queries);

/* Number of vertices / faces / boundary edges (directed edges with nonzero net
 * multiplicity over the faces; 0 for a closed, consistently oriented mesh) of a
 * mesh (-1 if mesh is NULL, or if the host memory to find the boundary edges,
 * which the first call does, is missing). */
int64_t dv_mesh_num_verts(const dv_mesh *mesh);
int64_t dv_mesh_num_faces(const dv_mesh *mesh);
int64_t dv_mesh_num_boundary_edges(const dv_mesh *mesh);
/* Number of strip events of the mesh's visiting order (dv_build_strips; nf
 * <= events <= 3 nf), the unit the forward and FP64 passes walk per query; -1
 * if mesh is NULL. */
int64_t dv_mesh_num_strip_events(const dv_mesh *mesh);

/* Synchronize `stream` and report (then clear) the sticky device error word
 * of the mesh: DV_ERR_TIMEOUT if a kernel's bounded wait ran out. */
dv_status dv_mesh_check(dv_mesh *mesh, void *stream);

/* Free the mesh and its scratch, in stream order on the stream of the mesh's
 * most recent call (cudaFreeAsync: no device-wide wait). Work that uses the mesh
 * on any other stream must be complete, or ordered before that stream, first.
 * NULL is a no-op. */
void dv_mesh_destroy(dv_mesh *mesh);

/* Winding numbers w(q), Eq. (5), for either
 *   - an explicit query list: d_queries float32 [nq][3] (grid must be NULL), or
 *   - the voxel centres of *grid (d_queries must be NULL, nq = nx*ny*nz or 0).
 * d_out_w float32 [nq]. `prec` as above. Stream-ordered, no sync. */
dv_status dv_winding(const dv_mesh *mesh, const float *d_queries, int64_t nq, const dv_grid *grid, float *d_out_w,
                     dv_precision prec, void *stream);

/* Voxelization (Algorithm 1 over a grid, §3): occupancy uint8 [nx*ny*nz]
 * (1 where w > 0.5, else 0) and optionally w itself (d_out_w may be NULL).
 * If report is non-NULL the call synchronizes `stream` and fills it. */
dv_status dv_voxelize_grid(const dv_mesh *mesh, const dv_grid *grid, float *d_out_w, uint8_t *d_out_occ,
                           dv_precision prec, dv_report *report, void *stream);

/* Adjoint: d_dverts float32 [nv][3] is OVERWRITTEN with
 *     sum_q d_upstream[q] * dw(q)/dV,
 * the derivative of Eq. (5) with Eq. (7) (the paper claims differentiability,
 * §1 and §2.4, but gives no formula). Every (query, face) pair is evaluated:
 * each face's derivative is summed over its three directed edges p -> r
 * (a = p - q, b = r - q): dOmega/dp += (b x a) / (|a| (|a||b| + a.b)),
 * dOmega/dr += (b x a) / (|b| (|a||b| + a.b)), equal to the chain rule through
 * Eq. (7) for q off the face; the terms of an edge whose segment contains the
 * query (the derivative does not exist there) are skipped. Queries as in
 * dv_winding (list or grid), d_upstream float32 [nq]. FP32 per-pair arithmetic
 * (|a||b| + a.b formed without cancellation near an edge segment), FP64
 * cross-block reduction; deterministic (no floating-point atomics).
 * Stream-ordered, no sync. */
dv_status dv_winding_backward(const dv_mesh *mesh, const float *d_queries, int64_t nq, const dv_grid *grid,
                              const float *d_upstream, float *d_dverts, void *stream);

/* The same adjoint as dv_winding_backward (same arguments, same result up to
 * FP32 rounding, for queries off the mesh), computed from the mesh's boundary
 * curve: the solid angle of a surface depends only on its boundary, so summed
 * over the faces the derivative of Eq. (7) cancels on every edge shared by two
 * consistently oriented faces. What remains is, per directed edge p -> r with
 * net multiplicity m and a = p - q, b = r - q,
 *     dOmega/dp = m (b x a) / (|a| (|a||b| + a.b)),
 *     dOmega/dr = m (b x a) / (|b| (|a||b| + a.b)),
 * one evaluation per (boundary edge, query) instead of per (face, query). The
 * gradient is exactly 0 for a closed mesh and off the boundary vertices. A
 * query on a boundary edge (|a||b| + a.b = 0) contributes nothing. No
 * counterpart in the paper: an evaluation of the same derivative. FP32 pair
 * arithmetic, FP64 vertex gather in a fixed order (deterministic).
 * Stream-ordered, no sync; the first call on a mesh also finds its boundary
 * edges on the host and uploads them (pageable copies). */
dv_status dv_winding_backward_boundary(const dv_mesh *mesh, const float *d_queries, int64_t nq, const dv_grid *grid,
                                       const float *d_upstream, float *d_dverts, void *stream);

/* No counterpart in the paper: a service of this library.
 * Winding numbers of the voxel centres of *grid (as dv_winding with
 * DV_PREC_FP32_KAHAN) for a mesh given directly as d_verts float32 [nv][3] and
 * d_faces int32 [nf][3], written to d_out_w float32 [nx*ny*nz], with NO device
 * allocation by the library: no dv_mesh is created, and no cudaMalloc, cudaFree
 * or other allocating call is made. It is meant for callers that cannot let a
 * library allocate: a process whose own allocator or memory budget already owns
 * the device memory (for example a server that has divided it among requests),
 * or a loop that cannot afford the device-wide synchronization that cudaMalloc
 * and cudaFree may cause.
 * The library's working memory on this path (packed face records, per-split
 * partial sums, an error word) is one fixed 32 MiB array compiled into the
 * library; a GPU on which the library's code is loaded keeps it until the
 * process exits. Requests that need more (about 48 bytes per face, plus 8 bytes
 * per query times the number of face splits for small grids) are rejected with
 * DV_ERR_UNSUPPORTED and a message giving the sizes. The first call on a device
 * looks up that array's device address (cudaGetSymbolAddress, no allocation);
 * make that first call before any stream capture. Every call on a device uses
 * the same array, so calls that overlap on the GPU (other streams, other host
 * threads) race and corrupt each other; serialize them. Faces are checked on the
 * device: an index outside [0, nv) gives DV_ERR_INVALID_MESH. The call
 * SYNCHRONIZES `stream` once, at the end, to read that check. */
dv_status dv_winding_grid_noalloc(const float *d_verts, int64_t nv, const int32_t *d_faces, int64_t nf,
                                  const dv_grid *grid, float *d_out_w, void *stream);

/* One request of a batch: the voxelization of a resident mesh over a grid
 * (occupancy, optionally w) and, if d_upstream is set, its adjoint. */
typedef struct {
    const dv_mesh *mesh;
    dv_grid grid;
    float *d_out_w;          /* float32 [nx*ny*nz] or NULL */
    uint8_t *d_out_occ;      /* uint8 [nx*ny*nz], required */
    const float *d_upstream; /* float32 [nx*ny*nz] or NULL (no adjoint) */
    float *d_dverts;         /* float32 [nv][3], overwritten; required with d_upstream */
} dv_request;

/* Run n independent requests (each as dv_voxelize_grid + dv_winding_backward would)
 * as ONE CUDA graph launched on `stream`: the library captures one parallel
 * branch per request, so the work of different requests overlaps on the GPU,
 * then launches the graph and returns without waiting. Each request's results
 * are identical to running it alone (same kernels, same launch plans). Used by
 * the request server (continuous batching). Scratch is reserved on `stream`
 * before capture; the meshes must not be used by other work until the batch is
 * done, and a mesh may appear only once per batch. `stream` must be a created
 * stream: the legacy and per-thread default streams cannot be captured and are
 * rejected with DV_ERR_INVALID_ARG. Host calls are serialized by a lock. No
 * counterpart in the paper (serving is this library's addition). */
dv_status dv_run_batch(const dv_request *reqs, int n, dv_precision prec, void *stream);

/* Eq. (4), the naive dipole discretization used by the paper for mesh morphing
 * (§2.4: the exact winding number is almost binary, so its gradient vanishes):
 *     W_dip(q) = (1/4pi) sum_f <n_f, (c_f - q)/|c_f - q|^3> Delta_f,
 * c_f the face centroid, n_f its unit outward normal, Delta_f its area; a query at
 * a centroid gets 0 from that face. Queries as in dv_winding; FP32 terms with
 * Kahan sums across face tiles. d_out_w float32 [nq]. Stream-ordered, no sync. */
dv_status dv_dipole_winding(const dv_mesh *mesh, const float *d_queries, int64_t nq, const dv_grid *grid,
                            float *d_out_w, void *stream);

/* Adjoint of dv_dipole_winding: d_dverts float32 [nv][3] OVERWRITTEN with
 * sum_q d_upstream[q] dW_dip(q)/dV (analytic; deterministic FP64 vertex gather). */
dv_status dv_dipole_backward(const dv_mesh *mesh, const float *d_queries, int64_t nq, const dv_grid *grid,
                             const float *d_upstream, float *d_dverts, void *stream);

/* Algorithm 2 (Flipping Duplication, §2.3): turn an open mesh into an almost
 * closed thin shell, Sigma^-2 = (V u V', F u F'), so that Algorithm 1 voxelizes
 * it like a closed mesh. d_verts float32 [nv][3] must be the vertices the mesh
 * was created or last updated with. Outputs (caller-owned, device):
 *   d_out_verts float32 [2nv][3]: V, then V' with v' = v - eps * N_v,
 *   d_out_faces int32  [2nf][3]: F, then F' = {(v0', v2', v1')} (reversed orientation).
 * N_v is the normalized sum of the incident faces' (v1-v0)x(v2-v0) (area-weighted;
 * the paper does not specify), summed in FP64 in a fixed order; a vertex with no
 * incident face keeps v' = v. The paper suggests eps = 0.01. Stream-ordered, no sync. */
dv_status dv_flipped_duplication(const dv_mesh *mesh, const float *d_verts, float eps, float *d_out_verts,
                                 int32_t *d_out_faces, void *stream);

/* Per-kernel timing of this library's own launches, for measurement tools.
 * dv_profile_enable(1) makes every later launch (on any stream) record a CUDA
 * event pair on its own stream; dv_profile_read synchronizes on those events and
 * copies up to `cap` entries: names[i] (static strings), total milliseconds,
 * launch counts. Returns the number of distinct kernels. dv_profile_enable(0)
 * stops recording; dv_profile_reset clears the totals. Not thread-safe. */
void dv_profile_enable(int on);
void dv_profile_reset(void);
int dv_profile_read(const char **names, double *total_ms, int64_t *launches, int cap);

/* Count of kernels this library has launched since load (all streams). */
int64_t dv_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* DV_API_H */
