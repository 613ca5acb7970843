/*
 * csm.h -- C ABI of the consistent cone-beam system-matrix projectors (sm_103a).
 *
 * The library applies the system matrix W of "Computation of a Consistent System Matrix
 * for Cone-beam Computed Tomography" without storing it: every entry W_ij is the exact
 * area (2D fan beam) or volume (3D circular cone beam) of the intersection of voxel j with
 * the cone from the source to detector element i (Introduction, Eq. (ip): p = W u), and is
 * evaluated on the fly from closed-form triangle / trapezoid atoms (2D, Sections
 * "Triangle", "Trapezoid", Eq. (2d procedure)) and from their 3D extension (Section "The
 * Three-dimensional Case", Eq. (rel vol 3d), Eq. (res vol 3d)).
 *
 * Geometry (Section "Notation and Setup", Eq. (z rotation)): the source sits at
 * (s cos phi, s sin phi, 0) and rotates about z; the flat detector lies at distance
 * sdd - s behind the isocentre, perpendicular to the source-isocentre ray.  A point P is
 * seen at detector coordinates u = sdd (-P_x sin phi + P_y cos phi) / t and
 * v = sdd P_z / t with depth t = s - P_x cos phi - P_y sin phi.  Detector corner k lies at
 * u_k = (k - nu/2) du + u_off (rows: v_l = (l - nv/2) dv + v_off); element k spans
 * [u_k, u_{k+1}].  The voxel grid is centred on the origin: voxel i spans
 * [(i - nx/2) a, (i + 1 - nx/2) a] (likewise y with b, z with c).
 *
 * Memory layouts (all contiguous, batch outermost, caller-owned device memory):
 *   volume    x[batch][nz][ny][nx]        (2D: nz = 1)
 *   sinogram  p[batch][n_views][nv][nu]   (2D: nv = 1)
 *
 * Every call is asynchronous on the given CUDA stream (NULL = legacy default stream).
 * A geometry belongs to the device that was current when it was created: csm_forward,
 * csm_back and csm_nnz return CSM_EINVAL when another device is current.
 * Argument errors are returned synchronously; a failed kernel launch returns
 * CSM_ECUDA.  Nothing aborts the process.  The library owns only the device geometry
 * table created by csm_geom_create_*; every other buffer (inputs, outputs, workspace)
 * belongs to the caller.
 */
#ifndef CSM_H_
#define CSM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct csm_geom_s* csm_geom_t;

typedef enum {
    CSM_OK = 0,
    CSM_EINVAL = 1,         /* bad argument (NULL pointer, size, dtype, workspace too small) */
    CSM_EGEOM = 2,          /* geometry not supported (e.g. source inside the grid's circle) */
    CSM_ENOMEM = 3,         /* the geometry table could not be allocated                    */
    CSM_ECUDA = 4,          /* a CUDA call failed; see csm_last_cuda_error()                 */
    CSM_EUNSUPPORTED = 5,   /* valid request that this build does not implement              */
    CSM_ETIMEOUT = 6        /* a bounded device-side wait gave up                            */
} csm_status;

typedef enum { CSM_F32 = 0, CSM_F64 = 1, CSM_BF16 = 2, CSM_F16 = 3 } csm_dtype;

/* flags for csm_forward / csm_back */
#define CSM_ACCUMULATE        1   /* add into the output instead of overwriting it           */
#define CSM_RELATIVE_WEIGHTS  2   /* entries divided by the voxel measure ab (abc), as in the
                                     paper's A_3, A_4, Vol_rel                                */
#define CSM_VOXEL_DRIVEN      4   /* forward only: the voxel-driven scatter variant (the form of
                                     the paper's Algorithm 1): shared-memory partial sums of
                                     detector elements per CTA, then global atomics; FP sums in
                                     no fixed order; workspace from csm_workspace_bytes(op = 2) */
#define CSM_EXPORT_TRANSPOSE  8   /* csm_export_csr: rows are voxels (the CSR of W^T)         */

/* 2D fan-beam geometry.  angles == NULL means phi_v = 2 pi v / n_views. */
typedef struct {
    int nx, ny;              /* pixel grid                                     */
    double a, b;             /* pixel sides in x, y                            */
    int n_views;             /* number of gantry angles                        */
    const double* angles;    /* host array of n_views angles [rad] or NULL     */
    double s;                /* source - isocentre distance                    */
    double sdd;              /* source - detector distance s + d               */
    int nu;                  /* detector elements                              */
    double du;               /* element width d_y                              */
    double u_off;            /* detector shift along u                         */
} csm_geom2d_desc;

/* 3D circular cone-beam geometry (rotation about z). */
typedef struct {
    int nx, ny, nz;
    double a, b, c;
    int n_views;
    const double* angles;
    double s, sdd;
    int nu, nv;              /* detector columns (u) and rows (v)              */
    double du, dv;           /* element sizes d_y, d_z                         */
    double u_off, v_off;
} csm_geom3d_desc;

/* Validate a 2D geometry and build its device table (Eq. (beta_computation): the rays to
 * the detector corners; Appendix Eq. (y expression), Eq. (x expression): each corner ray
 * as a line across the pixel grid).  Requires s > the grid's circumradius and sdd > s
 * (the cone lies between source and detector), positive sizes.  Must be called with the
 * target device current.  On success *out owns device memory until csm_geom_free.
 * Errors: CSM_EINVAL (NULL / non-positive sizes), CSM_EGEOM, CSM_ENOMEM, CSM_ECUDA. */
csm_status csm_geom_create_2d(const csm_geom2d_desc* desc, csm_geom_t* out);

/* Same for the 3D geometry (Section "The Three-dimensional Case").  Also CSM_EUNSUPPORTED
 * when the largest footprint of one voxel in a view exceeds the kernels' per-voxel slots
 * (its height over dv, plus 3, above 8 row corners; its width over du, rounded down, plus 1
 * above 6 crossing corner lines), or when nv * nu >= 2^31. */
csm_status csm_geom_create_3d(const csm_geom3d_desc* desc, csm_geom_t* out);

/* Release the geometry (synchronises its device with cudaFree; the table is released on the
 * device that holds it and the caller's current device is restored).  NULL is ignored. */
void csm_geom_free(csm_geom_t geom);

/* Per-element detector sensitivity weights (gains), the measurement model p_i = w_i (W x)_i
 * (the paper's element-wise measurement of Section "Notation and Setup" with a detector whose
 * elements respond differently).  weights: host array of n_views x nv x nu values (nv = 1 in
 * 2D) in the layout of p, finite; NULL removes them (all 1).  From then on csm_forward
 * multiplies each element's value by its weight, csm_back projects diag(w) p (so it stays
 * the adjoint), and csm_export_csr scales the rows of W; csm_nnz and the line-based
 * comparators are unaffected.  Copies the weights to memory owned by the geometry on its
 * device (synchronous).  Errors: CSM_EINVAL (NULL geometry, non-finite weight, another device
 * current), CSM_ENOMEM, CSM_ECUDA. */
csm_status csm_geom_set_element_weights(csm_geom_t geom, const double* weights);

/* Bytes of caller-provided device workspace that csm_forward / csm_back need for this
 * geometry, batch and arithmetic type (op: 0 = forward, 1 = back, 2 = forward with
 * CSM_VOXEL_DRIVEN, 3 = back into an x stored in another type than the arithmetic, e.g. BF16
 * or F16: op 1's workspace and, in 3D, an FP32 / FP64 copy of a chunk of x in which the sums
 * are formed before x is written, rounded once; csm_back accepts op 1's size too and then
 * runs the 3D back projection in one launch over all views).  The workspace holds the
 * batch-interleaved copies of the input that the kernels gather from (and the voxel-driven
 * forward's sums). */
csm_status csm_workspace_bytes(csm_geom_t geom, int op, int64_t batch, csm_dtype compute,
                               size_t* bytes);

/* p = W x  (Algorithm 1, "Computation of W in 2D", and its 3D counterpart).
 *   x : device pointer, x_dt elements, layout x[batch][nz][ny][nx]
 *   p : device pointer, p_dt elements, layout p[batch][n_views][nv][nu]
 *   Arithmetic is FP64 when x_dt or p_dt is CSM_F64, else FP32 (BF16/F16 are storage
 *   types only).  workspace: device pointer of at least csm_workspace_bytes(op = 0);
 *   may alias neither x nor p.  Returns CSM_EINVAL when the workspace is too small.
 *   Ray-driven gather: each element of p is written once, summed in a fixed order
 *   (bit-reproducible) -- in 3D wherever neighbouring row planes lie farther apart than twice
 *   a plane's height change across a voxel (as in the 128^3 and 512^3 cone-beam geometries);
 *   elsewhere the 3D forward adds a row's entries through shared-memory atomics of one warp
 *   and its FP32 sums may differ in the last bits between runs.  With CSM_VOXEL_DRIVEN: the
 *   scatter variant. */
csm_status csm_forward(csm_geom_t geom, const void* x, void* p, int64_t batch,
                       csm_dtype x_dt, csm_dtype p_dt, int flags,
                       void* workspace, size_t workspace_bytes, void* cuda_stream);

/* x = W^T p, the adjoint of csm_forward with the same entries (Section "Algorithm 1" and
 * the paper's adjoint-mismatch check, Section "Numerical Experiments").  Gather form (one
 * thread per two neighbouring pixels in 2D, one lane per voxel in 3D, where the voxel's value is summed by
 * parts over a differenced sinogram), fixed summation order, no atomics.
 * Arguments as for csm_forward with the roles of x and p exchanged (workspace from
 * csm_workspace_bytes(op = 1); with x stored in another type than the arithmetic, op = 3
 * gives the faster form in 3D, see there). */
csm_status csm_back(csm_geom_t geom, const void* p, void* x, int64_t batch,
                    csm_dtype p_dt, csm_dtype x_dt, int flags,
                    void* workspace, size_t workspace_bytes, void* cuda_stream);

/* Number of nonzero entries of W for this geometry: (voxel, view, element) whose
 * intersection exceeds 1e-6 of the voxel's area / volume (the resolution of the FP32
 * evaluation), computed once on the device and cached.  Synchronises the stream. */
csm_status csm_nnz(csm_geom_t geom, int64_t* nnz, void* cuda_stream);

/* ---- vector kernels of the reconstruction solvers -------------------------------------
 * The paper reconstructs by Nesterov's accelerated gradient on the Tikhonov objective with W
 * normalised by its spectral norm from 100 power iterations (Section "Numerical
 * Experiments", Eq. (exp_tikh)), and names the conjugate-gradient method in the same
 * section.  These kernels keep every scalar of such an iteration in device memory. */

/* Bytes of workspace csm_dot needs for `batch` inner products. */
csm_status csm_dot_workspace_bytes(int64_t batch, size_t* bytes);

/* out[b] = sum_i a[b n + i] * c[b n + i] for b < batch (1 <= batch <= 65535): FP64
 * accumulation, fixed summation order (bit-reproducible).  a, c: device arrays of dtype dt;
 * out: device array of `batch` doubles; workspace: device scratch of
 * csm_dot_workspace_bytes(batch) bytes, contents on return unspecified. */
csm_status csm_dot(const void* a, const void* c, int64_t n, int64_t batch, csm_dtype dt,
                   double* out, void* workspace, size_t workspace_bytes, void* cuda_stream);

/* y[b n + i] = A_b x[b n + i] + B_b y[b n + i] with per-item coefficients
 *   A_b = a_c * a_num[b] / a_den[b],  B_b = b_c * b_num[b] / b_den[b]
 * where a NULL num / den device pointer stands for 1 and a zero denominator gives 0.
 * flags bit 0 (bit 1): use sqrt(a_den[b]) (sqrt(b_den[b])).  x may be NULL (then A_b x = 0);
 * when B_b is 0, y is not read.  In place on y (dtype dt). */
csm_status csm_axpby(int64_t n, int64_t batch, csm_dtype dt, double a_c, const double* a_num,
                     const double* a_den, const void* x, double b_c, const double* b_num,
                     const double* b_den, void* y, int flags, void* cuda_stream);

/* The momentum of Nesterov's method (FISTA form, t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2,
 * theta_k = (t_k - 1) / t_{k+1}) for a batch whose items are at different iterations, as in a
 * reconstruction server that lets new requests join a running batch: item b reads
 * theta = theta_table[k[b]] (0 for k[b] outside 0 .. n_table - 1), writes one_plus_theta[b] =
 * 1 + theta and theta[b] = theta, and increments k[b].  All device arrays (k: int32, the rest
 * float64); theta_table may be NULL when n_table is 0.  Asynchronous on the stream, so an
 * iteration can be captured in a CUDA graph and replayed while items come and go. */
csm_status csm_fista_coeffs(int64_t batch, const double* theta_table, int n_table, int32_t* k,
                            double* one_plus_theta, double* theta, void* cuda_stream);

/* out[i] = num[i] / den[i] for i < n, and 0 where den[i] == 0 (dt = CSM_F32 or CSM_F64; device
 * arrays, out may alias num).  The data scaling of SART (the measured projections divided by
 * the row sums of W).  Asynchronous on the stream. */
csm_status csm_ediv(int64_t n, csm_dtype dt, const void* num, const void* den, void* out,
                    void* cuda_stream);

/* csm_dot without a workspace argument, for callers that cannot allocate device memory
 * (e.g. everything is owned by a pool allocator, a plug-in given no allocator, or a loop
 * where the device synchronisation cudaMalloc / cudaFree may cause is not acceptable).  The
 * paper has no counterpart: this is an interface for such callers only.  The partial sums
 * go to a fixed 128 KiB array in the library's device memory (held on every GPU that loads
 * the library until exit), so batch may not exceed CSM_DOT_NOALLOC_MAX_BATCH: larger
 * batches return CSM_EINVAL.  Result and arguments otherwise as csm_dot (same kernels, same
 * summation order).  The first call on a device looks up the array's device address with
 * that device current (and caches it with the identifier of the device's CUDA context, so a
 * call after cudaDeviceReset looks it up again); make that first call before any stream
 * capture.  All calls share the
 * one array: calls that may overlap on the GPU (different streams, or different host
 * threads) race and must be serialised by the caller.  No allocation is made. */
#define CSM_DOT_NOALLOC_MAX_BATCH 64
csm_status csm_dot_noalloc(const void* a, const void* c, int64_t n, int64_t batch, csm_dtype dt,
                           double* out, void* cuda_stream);

/* ---- measurement ----------------------------------------------------------------------
 * The paper has no counterpart: this measures the roofline that bounds the projectors.
 * Their entries are geometry evaluated with plain FP32 (FP64) arithmetic, so the binding
 * peak is the device's fused multiply-add issue rate, measured here rather than assumed.
 *
 * Runs `launches` back-to-back launches of a kernel of independent FMA chains (dt CSM_F32
 * or CSM_F64; blocks_per_sm blocks of 256 threads on every SM, `iters` x 128 FMAs per
 * thread) on the stream, timed with CUDA events on that stream, and waits for it.  Returns
 * the flops executed (2 per FMA) and the elapsed seconds; their ratio is the peak at the
 * clocks the GPU ran meanwhile.  Allocates nothing.  Errors: CSM_EINVAL (non-positive
 * counts, other dtypes), CSM_ECUDA. */
csm_status csm_fma_rate(csm_dtype dt, int64_t iters, int blocks_per_sm, int launches,
                        double* flops, double* seconds, void* cuda_stream);

/* The paper has no counterpart: instrumentation.  Writes to *count the number of kernels this
 * library has launched from the host since it was loaded, on every device and stream (every
 * launch site increments one process-wide counter just before it launches).  Replays of a
 * CUDA graph that captured library launches are not counted again.  Differences of two
 * readings count the launches of the calls in between.  Errors: CSM_EINVAL (count NULL). */
csm_status csm_launch_count(uint64_t* count);

/* ---- line-based comparator projectors ----------------------------------------------------
 * The line-integration system matrices the paper compares the consistent one with (Section
 * "Related work": Siddon's and Joseph's methods among the line-based approaches; Section
 * "Computational complexity": "several lines per detector element, averaged"), on the same
 * geometry handle and layouts as csm_forward / csm_back:
 *   CSM_LINE_SIDDON  W_ij = length of the ray inside voxel j;
 *   CSM_LINE_JOSEPH  the ray sampled at the centre plane of every voxel slice along its major
 *                    axis, the volume interpolated linearly (2D) / bilinearly (3D) between
 *                    the voxel centres of the slice, weighted by the ray length per slice.
 * An element's value is the mean over `lines` rays (lines x lines in 3D) from the source to
 * evenly spaced points of the element, u = u_k + (m + 1/2) du / lines (1 <= lines <= 64).
 * csm_back_line is the exact adjoint of csm_forward_line (the same rays and weights), added
 * into x with atomics: x must be CSM_F32 or CSM_F64 (else CSM_EUNSUPPORTED); its FP sums are
 * in no fixed order.  flags: CSM_ACCUMULATE.  No workspace; asynchronous on the stream. */
#define CSM_LINE_SIDDON 1
#define CSM_LINE_JOSEPH 2
csm_status csm_forward_line(csm_geom_t geom, int model, int lines, const void* x, void* p,
                            int64_t batch, csm_dtype x_dt, csm_dtype p_dt, int flags,
                            void* cuda_stream);
csm_status csm_back_line(csm_geom_t geom, int model, int lines, const void* p, void* x,
                         int64_t batch, csm_dtype p_dt, csm_dtype x_dt, int flags,
                         void* cuda_stream);

/* ---- the system matrix as an explicit sparse matrix -------------------------------------
 * The paper writes the reconstruction problem with W as a matrix (Introduction, Eq. (ip):
 * p = W u) and names the algebraic row-action methods (ART, SART) among the reconstruction
 * methods.  For problems small enough to store W, csm_export_csr writes it in CSR form,
 * computed on the device from the same closed-form entries as csm_forward / csm_back.
 *
 * Rows are detector elements, row index (view nv + l) nu + k, columns voxels (x layout
 * index); with CSM_EXPORT_TRANSPOSE rows are voxels and columns elements (the CSR of W^T).
 * Column indices are sorted within each row.  Stored entries are those whose value exceeds
 * the resolution of the arithmetic: 1e-6 of the voxel's area / volume for CSM_F32 values (the
 * entries csm_nnz counts), 1e-12 for CSM_F64; values are areas / volumes, or fractions of
 * the voxel with CSM_RELATIVE_WEIGHTS.  flags: CSM_EXPORT_TRANSPOSE | CSM_RELATIVE_WEIGHTS.
 *   row_ptr : device array of n_rows + 1 int64 (n_rows = voxels or views x nv x nu), written
 *   col_idx, val : device arrays of `capacity` entries (int32, val_dt = CSM_F32 or CSM_F64);
 *             both NULL: only row_ptr and *nnz are computed
 *   nnz     : host pointer, receives the number of stored entries
 *   workspace : device scratch of csm_export_workspace_bytes(geom, flags) bytes
 * Synchronises the stream.  Errors: CSM_EINVAL (NULL pointers, capacity < *nnz (with *nnz
 * set), workspace too small, another device current), CSM_EUNSUPPORTED (2^31 or more rows or
 * columns), CSM_ECUDA. */
csm_status csm_export_workspace_bytes(csm_geom_t geom, int flags, size_t* bytes);
csm_status csm_export_csr(csm_geom_t geom, int flags, csm_dtype val_dt, int64_t* row_ptr,
                          int32_t* col_idx, void* val, int64_t capacity, int64_t* nnz,
                          void* workspace, size_t workspace_bytes, void* cuda_stream);

/* y = alpha A x + beta y for a CSR matrix A with n_rows rows (row_ptr int64, col_idx int32,
 * val / x / y device arrays of dt = CSM_F32 or CSM_F64), a warp per row summing in a fixed
 * order (bit-reproducible); beta = 0 does not read y.  With the CSR of W this is the forward
 * projection, with the CSR of W^T the back projection.  Asynchronous on the stream. */
csm_status csm_csr_spmv(int64_t n_rows, const int64_t* row_ptr, const int32_t* col_idx,
                        const void* val, csm_dtype dt, double alpha, const void* x,
                        double beta, void* y, void* cuda_stream);

/* Divides each row of a CSR matrix (values val, dt = CSM_F32 or CSM_F64) by its sum, in
 * place; rows summing to 0 are left unchanged.  row_sums: NULL or a device array of n_rows
 * values of dt receiving the sums.  The row and column normalisations of SART (W divided by
 * its row sums, W^T by the column sums of W).  Asynchronous on the stream. */
csm_status csm_csr_normalize_rows(int64_t n_rows, const int64_t* row_ptr, void* val,
                                  csm_dtype dt, void* row_sums, void* cuda_stream);

/* Waits for the stream and reports an asynchronous kernel failure as CSM_ECUDA. */
csm_status csm_sync_status(void* cuda_stream);

const char* csm_status_string(csm_status status);
/* Text of the last CUDA error seen by the library in this thread ("" if none). */
const char* csm_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CSM_H_ */
