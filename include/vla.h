/*
 * vla.h -- C ABI of libvla: page-wise tiny-matrix algebra and P1/P2 simplex
 * stiffness/mass assembly into CSR on one NVIDIA GB300 (sm_103a).
 *
 * Method: "On a vectorized basic linear algebra package for prototyping codes
 * in MATLAB", arXiv:2404.16039.  Each entry point names the passage that
 * defines the operation it computes.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Status: every call returns vla_status.  0 is success, > 0 a warning, < 0
 *    an error.  No call aborts, traps or throws across the ABI.  The message
 *    of the most recent failure on the calling host thread is available from
 *    vla_last_error().
 *  - Memory: unless a parameter says "host", every array pointer is a DEVICE
 *    pointer owned by the caller, on the current CUDA device.  The library
 *    never frees caller memory.  Handles (vla_mesh) own the device memory they
 *    allocate and release it in their destroy call.
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy
 *    default stream).  Work is enqueued on it; calls return without waiting
 *    unless stated otherwise.  Outputs are valid once the stream reaches them.
 *  - Indices are 0-based int32.  Counts above 2^31-1 are rejected with
 *    VLA_ERR_INVALID_ARG.
 *  - Page arrays (the paper's "am"/"av"/"as" arrays, Section 2.4) hold N small
 *    matrices.  VLA_LAYOUT_PAGE: an n x m x N array in column-major order, so
 *    entry (r, c) of page k is at k*n*m + r + c*n (each page contiguous, the
 *    MATLAB layout).  VLA_LAYOUT_SOA: entry (r, c) of page k is at
 *    (r + c*n)*N + k (page index fastest).  Vectors are n x N (page layout:
 *    k*n + r; SoA: r*N + k); scalars are N contiguous values.
 *  - Mesh arrays (Section 3, "coords" and "elems"): coords is dim x nn FP64
 *    column-major (node i's coordinates contiguous: coords[i*dim + d]);
 *    elems is nlb x ne int32 column-major (element k's nodes contiguous:
 *    elems[k*nlb + j]), nlb = dim+1 for P1 and (dim+1)(dim+2)/2 for P2.  P2
 *    local numbering: vertices first, then mid-edge nodes in the order
 *    2-D (1,2),(2,3),(1,3); 3-D (1,2),(2,3),(1,3),(1,4),(2,4),(3,4)
 *    (1-based local vertices).
 */
#ifndef VLA_H
#define VLA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t vla_status;

enum {
    VLA_OK = 0,
    VLA_WARN_SINGULAR = 1,     /* some pages/elements had det == 0 (IEEE inf/nan in their outputs) */
    VLA_PENDING = 2,           /* a server request is not finished yet (vla_server_poll) */
    VLA_ERR_INVALID_ARG = -1,  /* bad size, null pointer, unsupported shape or flag */
    VLA_ERR_INDEX_OOB = -2,    /* an element or facet references a node outside [0, nn) */
    VLA_ERR_OOM = -3,          /* device allocation failed */
    VLA_ERR_CUDA = -4,         /* a CUDA runtime call failed (message has the CUDA error) */
    VLA_ERR_TIMEOUT = -5,      /* a bounded wait expired */
    VLA_ERR_BUDGET = -6,       /* request exceeds the configured memory budget */
    VLA_ERR_DEGENERATE = -7,   /* an element repeats a node, or a facet has no owning element */
    VLA_ERR_UNSUPPORTED = -8   /* mesh outside the implemented limits (row length, element count) */
};

enum { VLA_F32 = 0, VLA_F64 = 1 };                      /* dtype */
enum { VLA_LAYOUT_PAGE = 0, VLA_LAYOUT_SOA = 1 };        /* page-array layout */
enum { VLA_P1 = 1, VLA_P2 = 2 };                         /* element order */
enum { VLA_PREC_FP64 = 0, VLA_PREC_MIXED = 1 };          /* assembly precision */
enum { VLA_COEFF_POLY = 0, VLA_COEFF_EXP = 1,            /* coefficient kind (see vla_assemble) */
       VLA_COEFF_POLY_IP = 2, VLA_COEFF_EXP_IP = 3 };

/* Library version, 100*major + minor (housekeeping; no counterpart in the
 * paper).  Cannot fail. */
int32_t vla_version(void);

/* Copies the last error message of the calling thread into buf (NUL
 * terminated, truncated to len).  Returns the full message length. */
size_t vla_last_error(char *buf, size_t len);

/* ------------------------------------------------------------------------ */
/* Page primitives (the vectorization library of Section 2.4)               */
/* dtype: VLA_F32 or VLA_F64 (all arrays of the call share it).  Shapes      */
/* p, m, n in {2, 3}.  N >= 0; N == 0 is a no-op.  Arrays must not overlap.  */
/* ------------------------------------------------------------------------ */

/* amtam: C_k = A_k^T B_k for every page k.  A: p x m x N, B: p x n x N,
 * C: m x n x N.  (Section 2.4 lists amtam as the product of one page array
 * with the transpose of another and identifies it with MATLAB's pagemtimes
 * with the transpose flag on the first operand; its use on two gradient
 * pages in the P1 stiffness code of Section 3.5 fixes the reading A^T B.)
 * Errors: VLA_ERR_INVALID_ARG for an unknown dtype or layout, N < 0, a shape
 * outside the limits or a null array with N > 0; VLA_ERR_CUDA if a launch
 * fails. */
vla_status vla_amtam(int32_t dtype, int32_t layout, int64_t N, int32_t p, int32_t m, int32_t n, const void *A,
                     const void *B, void *C, void *stream);

/* astam: C_k = s_k A_k (page-wise scalar multiplication Id (x) pi, Section
 * 2.2 and the astam example of Section 2.4).  s: N scalars, A and C m x n x N.
 * Errors as for vla_amtam. */
vla_status vla_astam(int32_t dtype, int32_t layout, int64_t N, int32_t m, int32_t n, const void *s, const void *A,
                     void *C, void *stream);

/* avtam: y_k = v_k^T A_k (row vector times page, Section 2.4).  v: p x N,
 * A: p x n x N, y: n x N.  Errors as for vla_amtam. */
vla_status vla_avtam(int32_t dtype, int32_t layout, int64_t N, int32_t p, int32_t n, const void *v, const void *A,
                     void *y, void *stream);

/* amdet: det_k = det(A_k), signed (page-wise determinant det_W of Section
 * 2.3; the signed value -25/64 * 6 of the Section 3.2 example).  A: n x n x N,
 * det: N values.  Errors as for vla_amtam. */
vla_status vla_amdet(int32_t dtype, int32_t layout, int64_t N, int32_t n, const void *A, void *det, void *stream);

/* aminv: Ainv_k = A_k^{-1} (page-wise inverse of Section 2.3, pageinv) and,
 * if det != NULL, det_k.  The paper defines the inverse only where det != 0;
 * a page with det == 0 gets IEEE inf/nan entries and is counted.
 * n_singular: NULL, or a DEVICE int64 that receives the number of singular
 * pages (overwritten, not accumulated).  Returns VLA_OK; singular pages are
 * reported through n_singular only (the count lives on the device).
 * Errors as for vla_amtam. */
vla_status vla_aminv(int32_t dtype, int32_t layout, int64_t N, int32_t n, const void *A, void *Ainv, void *det,
                     int64_t *n_singular, void *stream);

/* amt: C_k = A_k^T (page-wise transpose, pagemtranspose, Section 2.4 and the
 * transpose map of Section 2.2; the X3D = amt(Y3D) index pages of the
 * Section 3.5 listings).  A: m x n x N, C: n x m x N, m and n in {2, 3}.
 * Errors as for vla_amtam. */
vla_status vla_amt(int32_t dtype, int32_t layout, int64_t N, int32_t m, int32_t n, const void *A, void *C,
                   void *stream);

/* avtav: out_k = a_k^T b_k (page-wise dot product of two vector arrays,
 * Section 2.4).  a, b: n x N with n in {2, 3}; out: N values.  Errors as for
 * vla_amtam. */
vla_status vla_avtav(int32_t dtype, int32_t layout, int64_t N, int32_t n, const void *a, const void *b, void *out,
                     void *stream);

/* Products with one single matrix or vector (Section 2.4: the single object
 * is copied to every page and multiplied page-wise).  Page arrays as above
 * (column-major pages, page or SoA layout); the single object S (column-major)
 * or s is one DEVICE array of the same dtype shared by all pages; every
 * dimension in [1, 16].
 *   amsm:  C_k = A_k S,       A: m x p x N, S: p x n, C: m x n x N
 *          (X_ip = amsm(coords3D, ip) of Section 3.4; dphi = amsm(tjacinv, dshape) of Section 3.5)
 *   amsv:  y_k = A_k s,       A: m x n x N, s: n, y: m x N
 *          (f_elems = amsv(fip, w) of Section 3.4)
 *   smamt: C_k = S A_k^T,     S: m x p, A: n x p x N, C: m x n x N
 *          (tjac = smamt(dshape, coords3D), the transposed Jacobian of Section 3.5)
 *   svamt: y_k = s^T A_k^T,   s: n, A: m x n x N, y: 1 x m x N (the values of amsv as rows)
 * Errors as for vla_amtam (every dimension must lie in [1, 16]). */
vla_status vla_amsm(int32_t dtype, int32_t layout, int64_t N, int32_t m, int32_t p, int32_t n, const void *A,
                    const void *S, void *C, void *stream);
vla_status vla_amsv(int32_t dtype, int32_t layout, int64_t N, int32_t m, int32_t n, const void *A, const void *s,
                    void *y, void *stream);
vla_status vla_smamt(int32_t dtype, int32_t layout, int64_t N, int32_t m, int32_t p, int32_t n, const void *S,
                     const void *A, void *C, void *stream);
vla_status vla_svamt(int32_t dtype, int32_t layout, int64_t N, int32_t m, int32_t n, const void *s, const void *A,
                     void *y, void *stream);

/* ------------------------------------------------------------------------ */
/* Meshes and assembly (Sections 3.1-3.5)                                    */
/* ------------------------------------------------------------------------ */

typedef struct vla_mesh vla_mesh;

typedef struct {
    int32_t dim, order, nlb;
    int64_t nn, ne, nfb, nnz;
    int32_t max_row_len;     /* longest CSR row */
    int32_t n_tiles;         /* row tiles of the assembly kernel */
    int64_t device_bytes;    /* device memory held by the handle */
    int64_t tile_elems;      /* element computations per assembly (sum over tiles; >= ne) */
    int64_t n_codes;         /* contribution codes streamed per assembly (including padding) */
    int32_t tile_budget;     /* incidence budget the tiles were cut with */
    int32_t reserved;
    int64_t smem_bytes;      /* shared memory per CTA of the mixed-precision assembly launch */
} vla_mesh_info_t;

/* Ingests a simplicial mesh and builds, on the device, everything the
 * assembly needs: the CSR pattern of the sparse assembly of Section 3.5
 * (every (elems(k,i), elems(k,j)) pair, duplicates merged,
 * explicit zeros kept, columns ascending), node->element incidence, the row
 * tiles of the assembly kernel and the owner of every boundary facet.
 *   dim 2 or 3; order VLA_P1 or VLA_P2; nn, ne >= 1.
 *   coords: dim x nn FP64 (device); elems: nlb x ne int32 (device).
 *   P2 elements list the vertices, then the edge midpoints in the order
 *   (0,1), (1,2), (0,2)[, (0,3), (1,3), (2,3)]; the mesh must be conforming
 *   (every element holding an edge uses the same midpoint node for it).
 *   faces:  dim x nfb int32 (device) boundary facets given by vertex nodes
 *           (triangles in 3-D, edges in 2-D), any orientation; NULL if nfb 0.
 * Validation: node indices outside [0, nn) -> VLA_ERR_INDEX_OOB; an element
 * that repeats a node, or a facet no element owns -> VLA_ERR_DEGENERATE; a CSR
 * row longer than 255 entries or ne >= 2^27 -> VLA_ERR_UNSUPPORTED.
 * Synchronises `stream` (the build sizes depend on device results).  The
 * handle keeps its own copies of coords/elems/faces; the caller's arrays may
 * be freed afterwards. */
vla_status vla_mesh_create(int32_t dim, int32_t order, int64_t nn, int64_t ne, const double *coords,
                           const int32_t *elems, int64_t nfb, const int32_t *faces, void *stream, vla_mesh **out);

/* Fills *info (host struct): the sizes of the mesh and of the CSR pattern of
 * the Section 3.5 assembly, and the tiling (no counterpart in the paper).
 * Errors: VLA_ERR_INVALID_ARG for a NULL argument. */
vla_status vla_mesh_info(const vla_mesh *mesh, vla_mesh_info_t *info);

/* Copies the CSR pattern of the Section 3.5 sparse assembly to caller buffers
 * (device): row_ptr nn+1 int32, col_idx nnz int32.  Either may be NULL.
 * Errors: VLA_ERR_INVALID_ARG for a NULL mesh; VLA_ERR_CUDA if a copy fails. */
vla_status vla_mesh_csr(const vla_mesh *mesh, int32_t *row_ptr, int32_t *col_idx, void *stream);

/* The CSR pattern of the Section 3.5 sparse assembly without a copy: device
 * pointers to the mesh's own row_ptr (nn+1 int32) and col_idx (nnz int32).
 * They stay valid, read-only, until vla_mesh_destroy.
 * Errors: VLA_ERR_INVALID_ARG for a NULL argument. */
vla_status vla_mesh_csr_view(const vla_mesh *mesh, const int32_t **row_ptr, const int32_t **col_idx);

/* Assembles K and M (Section 3.5 stiffness and mass listings) into the
 * mesh's CSR pattern:
 *   K_ij = sum_k c_k int_{T_k} grad phi_i . grad phi_j,
 *   M_ij = sum_k c_k int_{T_k} phi_i phi_j,
 * where c_k is the coefficient evaluated at the vertex centroid x_c of T_k:
 *   VLA_COEFF_POLY: c = ca + cb |x_c|^2;  VLA_COEFF_EXP: c = ca exp(cb sum_d x_c,d).
 *   VLA_COEFF_POLY_IP, VLA_COEFF_EXP_IP (P1 only): the paper's literal P1
 *   listing -- the same functions evaluated at the points of the degree-2
 *   rule (gqo = 2) of every element: K_k = (sum_i w_i c(x_i)) |T| G^T G and
 *   M_k(p,q) = |T| sum_i w_i c(x_i) lambda_p(x_i) lambda_q(x_i); P2 meshes get
 *   VLA_ERR_UNSUPPORTED.  Batches, the server and vla_element_pages_static
 *   take the centroid kinds only.
 * P1 integrals are exact; P2 stiffness uses the 4-point rule (exact for the
 * quadratic integrand of affine elements) and P2 mass the exact reference
 * mass matrix.  Outputs (device, FP64, any may be NULL):
 *   K_vals, M_vals: nnz values in the mesh's CSR order;
 *   vol: ne element measures |det V_k| / dim! (Section 3.2 volume script);
 *   K_pages, M_pages: the element matrices K3D, M3D as nlb x nlb x ne
 *   column-major pages (second output of the Section 3.5 listings).
 * precision: VLA_PREC_FP64 computes everything in FP64.  VLA_PREC_MIXED
 *   forms element matrices in FP32 from coordinates stored as float pairs.
 *   The geometry of an element is first computed in plain FP32 (edge vectors
 *   rounded once, one FMA per cofactor, det as an FMA dot product), whose
 *   det is within 11u perm(|V|) of the exact one (u = 2^-24, perm the
 *   permanent of the absolute Jacobian).  Where |det| < perm(|V|)/4 (flat
 *   or sliver elements, where that bound exceeds 44u relative) the element
 *   is recomputed from error-free float-pair edge vectors with a compensated
 *   determinant (error about 2u relative plus O(u^2 perm)) and Kahan's FMA
 *   algorithm for the remaining cofactors.  Every CSR value is a compensated
 *   (float-float) sum converted to FP64 once.
 * If n_singular != NULL (device int64), it receives the number of elements
 * with det == 0.  Deterministic: the same inputs give bit-identical outputs. */
vla_status vla_assemble(const vla_mesh *mesh, int32_t coeff_kind, double ca, double cb, int32_t precision,
                        double *K_vals, double *M_vals, double *vol, double *K_pages, double *M_pages,
                        int64_t *n_singular, void *stream);

/* vla_assemble and vla_boundary of the same mesh in one launch (the Section
 * 3.5 assembly and the Section 3.2/3.4 boundary normals and areas): the
 * persistent assembly CTAs compute the mesh's boundary facets after their
 * row tiles, in the precision given, instead of a second kernel after the
 * assembly.  The outputs equal those of the two separate calls bit for bit.
 * normals (dim x nfb) and areas (nfb) as for vla_boundary; every other
 * argument as for vla_assemble.  A mesh without boundary facets is assembled
 * as by vla_assemble (normals and areas may then be NULL).  Errors: those of
 * vla_assemble, and VLA_ERR_INVALID_ARG for a NULL normals or areas on a mesh
 * with boundary facets. */
vla_status vla_assemble_with_boundary(const vla_mesh *mesh, int32_t coeff_kind, double ca, double cb,
                                      int32_t precision, double *K_vals, double *M_vals, double *vol,
                                      double *K_pages, double *M_pages, int64_t *n_singular, double *normals,
                                      double *areas, void *stream);

/* Boundary facets (Section 3.2 normals of boundary faces; the areas used by
 * the surface integrals of Section 3.4): for facet f with vertex nodes
 * (x1, x2[, x3]) the normal n = (x2-x1) x (x3-x1) (3-D) or the edge vector
 * rotated by -90 degrees (2-D), oriented away from the remaining vertex of
 * the owning element, normalised to unit length; areas[f] = |n|/2 (3-D) or
 * the edge length (2-D).  normals: dim x nfb FP64 (facet f at f*dim + d),
 * areas: nfb FP64 (device).  precision as in vla_assemble.  A mesh without
 * boundary facets is a no-op.  Errors: VLA_ERR_INVALID_ARG for a NULL mesh or
 * output or an unknown precision; VLA_ERR_CUDA if a launch fails. */
vla_status vla_boundary(const vla_mesh *mesh, int32_t precision, double *normals, double *areas, void *stream);

/* Unnormalised outer normals of all element facets,
 * normals3D_k = (vectors3D_k)^{-T} normalsRef (Section 3.2, with the normal
 * transform X = A^{-T} of Section 2.3).  vectors3D_k holds x_j - x_last as
 * columns; normalsRef columns are -e_1..-e_dim and (1,..,1); column j is the
 * normal of the facet opposite local vertex j.  normals: dim x (dim+1) x ne
 * FP64 column-major pages (device). FP64 arithmetic.  Errors:
 * VLA_ERR_INVALID_ARG for a NULL mesh or output; VLA_ERR_CUDA if a launch
 * fails. */
vla_status vla_simplex_normals(const vla_mesh *mesh, double *normals, void *stream);

/* Element pages and volumes without a mesh handle and without allocating.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory where they need element matrices (a heap
 * owned by another framework, allocator-free real-time loops, code that must
 * not create a persistent handle).  It computes what vla_assemble writes to
 * K_pages, M_pages and vol, bit for bit (the same element arithmetic, in
 * both precisions), for the centroid coefficient kinds VLA_COEFF_POLY and
 * VLA_COEFF_EXP (the literal-quadrature kinds are rejected with
 * VLA_ERR_INVALID_ARG), from the raw arrays: coords dim x nn FP64 and elems
 * nlb x ne int32 (device, layouts as for vla_mesh_create).  Element indices
 * are checked on the device before any coordinate is read: an element with
 * a node index outside [0, nn) is skipped, its pages and volume are set to
 * NaN, and it is counted; vla_element_pages_static_check reports the count
 * of the last call.
 * Scratch: the float-pair split of the coordinates used by VLA_PREC_MIXED is
 * kept in a fixed device array built into the library (8 MiB per GPU that
 * loads it, held until the process exits); nn above 262,144 is rejected with
 * VLA_ERR_BUDGET.  No cudaMalloc/cudaFree or allocating library call is made.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * Every call shares the one array and the skip counter (cleared at the start
 * of each call): calls that overlap on the GPU (different streams, or
 * different host threads) race and must be serialised by the caller.
 * Outputs (device, any may be NULL): K_pages, M_pages nlb x nlb x ne
 * column-major, vol ne, n_singular (device int64, overwritten).
 * Errors (before any work): VLA_ERR_INVALID_ARG for an unknown dim, order,
 * coefficient kind or precision, nn < 1, ne < 0, too many elements, NULL
 * mesh arrays with ne > 0 or a non-finite coefficient; VLA_ERR_BUDGET for
 * nn > 262,144; VLA_ERR_CUDA if a launch fails. */
vla_status vla_element_pages_static(int32_t dim, int32_t order, int64_t nn, int64_t ne, const double *coords,
                                    const int32_t *elems, int32_t coeff_kind, double ca, double cb, int32_t precision,
                                    double *K_pages, double *M_pages, double *vol, int64_t *n_singular, void *stream);

/* Reports how many elements the last vla_element_pages_static call on the
 * current device skipped for a node index outside [0, nn) (the paper has no
 * counterpart; index validation of the allocation-free path).  Copies the
 * device counter to *n_skipped (host, may be NULL) on `stream` and
 * synchronises it.  Returns VLA_ERR_INDEX_OOB if the count is nonzero,
 * VLA_ERR_CUDA if the copy fails, VLA_OK otherwise. */
vla_status vla_element_pages_static_check(int64_t *n_skipped, void *stream);

/* Row-block partition for assembly on several GPUs (the data-parallel
 * sharding of the Section 3.5 assembly: every element is independent, the
 * CSR sum is the one exchange step).  A GPU that owns the contiguous rows
 * [row_begin, row_end) needs every element with a node in that range; the
 * elements shared with neighbouring blocks (the halo) are duplicated, so each
 * GPU assembles complete rows and no reduction across GPUs is needed.
 * vla_partition_rows writes the ascending ids of those elements (any node,
 * P2 mid-edge nodes included, in the range) to elem_ids (device int32,
 * capacity ne, may be NULL to count only) and their number to *n_elems
 * (host).  elems: nlb x ne int32 as for vla_mesh_create (device); indices
 * are compared, never dereferenced.  Synchronises `stream`.  Errors:
 * VLA_ERR_INVALID_ARG for a NULL n_elems or elems, nlb outside [3, 10], ne
 * outside [0, 2^31-1] or a range with row_begin < 0 or row_end < row_begin
 * (an empty range gives 0 elements); VLA_ERR_CUDA if a launch or copy fails. */
vla_status vla_partition_rows(int32_t nlb, int64_t ne, const int32_t *elems, int32_t row_begin, int32_t row_end,
                              int32_t *elem_ids, int64_t *n_elems, void *stream);

/* A mesh handle for one row block (Section 3.5 assembly split by rows, see
 * vla_partition_rows): the sub-mesh of the elements with a node in
 * [row_begin, row_end) and of the boundary facets whose smallest node lies in
 * that range, with the global node numbering (coords and nn are the whole
 * mesh's).  Rows [row_begin, row_end) of its CSR pattern and of the K and M
 * values vla_assemble writes are exactly those rows of the whole mesh's
 * (same columns, same summation order, same bits); its other rows are
 * partial and belong to other blocks.  Arguments as vla_mesh_create plus the
 * block.  Synchronises `stream`.  Errors: those of vla_mesh_create, and
 * VLA_ERR_INVALID_ARG for a block that is empty, reaches outside [0, nn) or
 * holds no element's node. */
vla_status vla_mesh_create_rows(int32_t dim, int32_t order, int64_t nn, int64_t ne, const double *coords,
                                const int32_t *elems, int64_t nfb, const int32_t *faces, int32_t row_begin,
                                int32_t row_end, void *stream, vla_mesh **out);

/* Every facet of the mesh once (the faces behind the paper's normals of all
 * faces and its face counts, Section 3.2): facet j of element k is opposite
 * local vertex j, with the element's other vertex nodes in local order; a
 * facet shared by elements k < k' is listed with k, and the list is ordered
 * by (k, j).  Outputs (device, any may be NULL): faces dim x nf int32,
 * owner 2 x nf int32 (k, j), neighbor nf int32 (k', or -1 for a boundary
 * facet); *n_faces and *n_boundary (host) receive nf and the number of
 * boundary facets.  Call with NULL arrays first to learn nf.  Integer work,
 * deterministic; synchronises `stream`.  Unnormalised normals of all facets:
 * vla_simplex_normals, column j of element k's page.  Errors:
 * VLA_ERR_INVALID_ARG for a NULL mesh; VLA_ERR_OOM if scratch cannot be
 * allocated; VLA_ERR_CUDA if a launch fails. */
vla_status vla_mesh_facets(const vla_mesh *mesh, int32_t *faces, int32_t *owner, int32_t *neighbor, int64_t *n_faces,
                           int64_t *n_boundary, void *stream);

/* Housekeeping (no counterpart in the paper): releases the handle and its
 * device memory (stream-ordered on the stream the mesh was created with,
 * which is synchronised first).  The memory returns to the library's device
 * memory pool, which keeps up to min(8 GiB, 1/16 of the device) of freed
 * memory mapped for later builds (the environment variable VLA_POOL_KEEP, in
 * bytes, sets that amount when the pool is first used; 0 keeps none).  The
 * temporary buffers of mesh builds are not the mesh's: each host thread that
 * builds meshes keeps up to 512 MiB of them per device for its next build
 * (more is returned when a build ends), freed when the thread ends.  NULL
 * is a no-op; cannot fail. */
vla_status vla_mesh_destroy(vla_mesh *mesh);

/* Failure detection (no counterpart in the paper): reads and clears the
 * mesh's device error word, synchronising `stream`:
 * VLA_ERR_TIMEOUT if a bounded wait of a kernel on this mesh expired since
 * the last check (its outputs are then incomplete), else VLA_OK.  Kernels
 * never spin without a limit; an expired wait ends the kernel early and is
 * reported here rather than by a fault. */
vla_status vla_mesh_check(vla_mesh *mesh, void *stream);

/* ------------------------------------------------------------------------ */
/* Quadrature, integrals, load vector, energies (Sections 3.4, 3.5)          */
/* ------------------------------------------------------------------------ */

/* The quadrature rule of Gauss_points(gqo, sdim) (Section 3.4) on a simplex of
 * dimension sdim (1 segment, 2 triangle, 3 tetrahedron), degree of exactness
 * gqo = 1..3: barycentric points ip ((sdim+1) x nip, point q at
 * q*(sdim+1)) and weights w (nip) summing to 1 (intquad's weights of
 * Section 3.5 are these times 1/sdim!).  Host arrays of at least 8 points;
 * any may be NULL.  VLA_ERR_UNSUPPORTED for other degrees. */
vla_status vla_quad_rule(int32_t sdim, int32_t gqo, int32_t *nip, double *ip, double *w);

/* Quadrature points X_ip = amsm(coords3D, ip) (Section 3.4): for every element
 * (facets = 0) or every boundary facet (facets = 1) and every point q of the
 * degree-gqo rule, X(:, q, k) = sum_j ip(j, q) x_j.  X: dim x nip x n FP64
 * column-major (device), n = ne or nfb.  FP64 arithmetic.  Errors:
 * VLA_ERR_INVALID_ARG for a NULL mesh or output, or facets = 1 on a mesh
 * without boundary facets; VLA_ERR_UNSUPPORTED for a degree outside 1..3;
 * VLA_ERR_CUDA if a launch fails. */
vla_status vla_quad_points(const vla_mesh *mesh, int32_t gqo, int32_t facets, double *X, void *stream);

/* The GI function of Section 3.4: value = sum_k sizes_k sum_q w_q f(:, q, k).
 *   fip: d x nip x n FP64 (device) -- f at the points of n simplices;
 *   w: nip host weights (nip <= 8); sizes: n FP64 (device) element volumes or
 *   facet areas; normals: d x n (device) or NULL.
 * Without normals out[c] (device, d <= 4 values) is the integral of component
 * c; with normals out[0] is the flux sum_k sizes_k (avg_k f) . n_k.  The sum is
 * reduced in a fixed order (bit-reproducible).  Allocates stream-ordered
 * scratch.  Errors: VLA_ERR_INVALID_ARG for n < 0, nip outside [1, 8], d
 * outside [1, 4], NULL w or out, or NULL fip or sizes with n > 0;
 * VLA_ERR_OOM if the scratch cannot be allocated; VLA_ERR_CUDA if a launch
 * fails. */
vla_status vla_gi(int64_t n, int32_t nip, int32_t d, const double *fip, const double *w, const double *sizes,
                  const double *normals, double *out, void *stream);

/* Load vector of Section 3.5 (rhs_vectorP1; P2 alike):
 * b2D(j, k) = |T_k| sum_q w_q f(x_q) phi_j(ip_q) for the degree-gqo rule, then
 * b_i = the sum of b2D(j, k) over the entries with elems(k, j) = i, in a fixed
 * order (each node's incident elements ascending).  fip: nip x ne FP64 (device) -- f at the points given by
 * vla_quad_points(mesh, gqo, 0, ...).  b: nn (device) or NULL; b2D: nlb x ne
 * (device) or NULL (then scratch).  FP64.  Errors: VLA_ERR_INVALID_ARG for a
 * NULL mesh or fip; VLA_ERR_UNSUPPORTED for a degree outside 1..3;
 * VLA_ERR_OOM if the scratch cannot be allocated; VLA_ERR_CUDA if a launch
 * fails. */
vla_status vla_rhs(const vla_mesh *mesh, int32_t gqo, const double *fip, double *b, double *b2D, void *stream);

/* Local energies of Section 3.5 (eq. Jk_comps): with u_k the element's nodal
 * values of u (nn FP64, device),
 *   J_local(0,k) = u_k^T K_k u_k / 2,  J_local(1,k) = u_k^T M_k u_k / 2,
 *   J_local(2,k) = -b2D(:,k)^T u_k,
 * from the element pages of vla_assemble (K_pages, M_pages: nlb x nlb x ne) and
 * the element loads of vla_rhs (b2D: nlb x ne); any of the three may be NULL
 * (its energy is then 0).  J_local: 3 x ne (device) or NULL; J_total: 3 values
 * (device) or NULL -- the sums over elements, i.e. u^T K u / 2, u^T M u / 2 and
 * -b^T u, reduced in a fixed order.  FP64.  Errors: VLA_ERR_INVALID_ARG for a
 * NULL mesh or u; VLA_ERR_OOM if the scratch for J_total cannot be allocated;
 * VLA_ERR_CUDA if a launch fails. */
vla_status vla_energies(const vla_mesh *mesh, const double *u, const double *K_pages, const double *M_pages,
                        const double *b2D, double *J_local, double *J_total, void *stream);

/* out_k = v_k^T A_k w_k (Section 2.4, avtamav): v, w n x N, A n x n x N
 * (VLA_LAYOUT_PAGE, column-major pages) or the SoA layout; out N.  n <= 16.
 * Errors: VLA_ERR_INVALID_ARG for an unknown dtype or layout, N < 0, n outside
 * [1, 16] or a NULL array with N > 0; VLA_ERR_CUDA if a launch fails. */
vla_status vla_avtamav(int32_t dtype, int32_t layout, int64_t N, int32_t n, const void *v, const void *A,
                       const void *w, void *out, void *stream);

/* ------------------------------------------------------------------------ */
/* Batched assembly (Section 3.5 assembly over many meshes at once)          */
/* ------------------------------------------------------------------------ */
/* The paper assembles one mesh per call; a batch runs the same computation
 * as vla_assemble for many meshes of any element type (triangles or
 * tetrahedra, P1 or P2) in ONE persistent kernel launch: the row tiles of all
 * meshes form one work list, and each CTA streams tiles of whatever mesh
 * comes next.  Every mesh's outputs are bit-identical to vla_assemble on that
 * mesh alone (the summation order of every value depends only on the mesh). */

typedef struct vla_batch vla_batch;

typedef struct {
    const vla_mesh *mesh;      /* the mesh (handle from vla_mesh_create) */
    int32_t coeff_kind;        /* as in vla_assemble */
    int32_t reserved;          /* 0 */
    double ca, cb;
    double *K_vals, *M_vals;   /* nnz FP64 each (device), or NULL */
    double *vol;               /* ne FP64 (device), or NULL */
    double *K_pages, *M_pages; /* nlb x nlb x ne FP64 (device), or NULL */
} vla_batch_job_t;

typedef struct {
    int32_t count;             /* jobs */
    int32_t n_work;            /* row tiles over all jobs (work items of the launch) */
    int32_t grid;              /* persistent CTAs of the launch */
    int32_t ctas_per_sm;       /* tuned residency (0 = occupancy limit) */
    int64_t smem_bytes;        /* dynamic shared memory per CTA */
    int64_t elements;          /* sum of ne */
    int64_t tile_elems;        /* element computations per launch (>= elements) */
    int32_t graph;             /* 1 if runs replay a captured CUDA graph */
    int32_t split;             /* 1: one persistent kernel per element type; 0: one kernel for all */
} vla_batch_info_t;

#define VLA_BATCH_GRAPH 1      /* capture the launch into a CUDA graph at creation */
#define VLA_BATCH_FUSED 2      /* one persistent kernel for every element type */
#define VLA_BATCH_SPLIT 4      /* one persistent kernel per element type present, back to back */
#define VLA_BATCH_AUTOTUNE 8   /* time both forms at creation (runs the batch) and keep the faster */

/* Builds the job table and work list of a batch on the device (batching of
 * the Section 3.5 assembly; no counterpart in the paper).
 *   jobs: host array of count >= 1 jobs (copied; meshes must outlive the batch).
 *   precision: VLA_PREC_FP64 or VLA_PREC_MIXED, for every job.
 *   n_singular: device int64[count] receiving, per job, the number of
 *     elements with det == 0 (reset by every run), or NULL.
 *   flags: VLA_BATCH_GRAPH captures the reset and the kernel(s) once into a
 *     CUDA graph (each run is one graph launch).  The launch form: one
 *     persistent kernel whose CTAs take tiles of every element type
 *     (VLA_BATCH_FUSED: one launch, shared memory sized for the largest tile of
 *     any type), or one persistent kernel per element type present, each
 *     sized for its own type (VLA_BATCH_SPLIT); neither flag: split when every
 *     type has several waves of tiles, else fused; VLA_BATCH_AUTOTUNE: run
 *     both at creation and keep the faster.  Results do not depend on it.
 * Synchronises `stream`.  Errors: VLA_ERR_INVALID_ARG, VLA_ERR_OOM,
 * VLA_ERR_UNSUPPORTED (a tile larger than shared memory), VLA_ERR_CUDA. */
vla_status vla_batch_create(const vla_batch_job_t *jobs, int32_t count, int32_t precision, int64_t *n_singular,
                            int32_t flags, void *stream, vla_batch **out);

/* Replaces job `index`'s coefficient (Section 3.5.1 coefficients) and output
 * pointers (same mesh), stream ordered: runs enqueued on `stream` afterwards see the new job.
 * Errors: VLA_ERR_INVALID_ARG for a NULL batch or job, an index outside
 * [0, count), another mesh or an unknown coefficient kind; VLA_ERR_CUDA if
 * the launch that updates the device job table fails. */
vla_status vla_batch_set_job(vla_batch *batch, int32_t index, const vla_batch_job_t *job, void *stream);

/* Enqueues one Section 3.5 assembly of every job on `stream` (one persistent launch, or
 * one graph launch with VLA_BATCH_GRAPH).  Errors: VLA_ERR_INVALID_ARG for a
 * NULL batch; VLA_ERR_CUDA if the launch fails. */
vla_status vla_batch_run(vla_batch *batch, void *stream);

/* Fills *info (host struct): the batch's launch shape (no counterpart in the
 * paper).  Errors: VLA_ERR_INVALID_ARG for a NULL argument. */
vla_status vla_batch_info(const vla_batch *batch, vla_batch_info_t *info);

/* As vla_mesh_check, for the batch's own error word (no counterpart in the
 * paper).  Errors: VLA_ERR_TIMEOUT as described there; VLA_ERR_INVALID_ARG
 * for a NULL batch; VLA_ERR_CUDA if the read fails. */
vla_status vla_batch_check(vla_batch *batch, void *stream);

/* Frees the batch (housekeeping; no counterpart in the paper).  No run of it
 * may still be in flight.  NULL is a no-op; cannot fail. */
vla_status vla_batch_destroy(vla_batch *batch);

/* One-shot batch of Section 3.5 assemblies: create, run once and free, all stream-ordered on `stream`
 * (no host synchronisation); the error word is not kept.  Errors: those of
 * vla_batch_create (flags 0), and VLA_ERR_CUDA if the launch fails. */
vla_status vla_batch_assemble(const vla_batch_job_t *jobs, int32_t count, int32_t precision, int64_t *n_singular,
                              void *stream);

/* ------------------------------------------------------------------------ */
/* Autotuning of the tile and warp mapping                                   */
/* ------------------------------------------------------------------------ */
/* The assembly maps elements to row tiles (the incidence budget bounds the
 * rows x incident elements of one tile, which sets the element records and
 * contribution lists a CTA holds in shared memory) and tiles to persistent
 * CTAs of 8 warps, each warp taking 32-pair chunks of a tile.  The tuner
 * times candidate budgets and CTA residencies on a sample mesh and keeps the
 * fastest for the element type and precision, process-wide: meshes built
 * afterwards use the tuned budget, and assemblies and batches the tuned
 * residency.  Results do not depend on either choice. */

typedef struct {
    int32_t tile_budget;       /* incidence budget of a row tile (0 = library default) */
    int32_t ctas_per_sm;       /* resident CTAs per SM (0 = occupancy limit) */
    double us;                 /* median time of one assembly of the sample mesh, microseconds (tuner output) */
} vla_tune_t;

/* Autotuner (no counterpart in the paper): times the Section 3.5 assembly of
 * vla_assemble (precision as given, coefficient 1 + |x|^2, K, M and vol
 * outputs, an L2 flush before every timed run) on the sample mesh for each
 * candidate budget (0.5x to 1.5x the default) and then each residency (1, 2,
 * 3, 4 and the occupancy limit) at the best budget, `reps` timed runs each
 * (median), stores the winner and returns it in *best.  The default budget and
 * the occupancy limit are timed first, and another candidate wins only when it
 * is at least 3 % faster.  coords/elems as for vla_mesh_create.  Allocates
 * scratch; synchronises `stream`.  Errors: VLA_ERR_INVALID_ARG for a NULL
 * best, an unknown element type or precision; the errors of vla_mesh_create
 * for the sample mesh; VLA_ERR_OOM, VLA_ERR_CUDA. */
vla_status vla_autotune(int32_t dim, int32_t order, int32_t precision, int64_t nn, int64_t ne, const double *coords,
                        const int32_t *elems, int32_t reps, void *stream, vla_tune_t *best);

/* Autotuner state (no counterpart in the paper): reads or sets the stored
 * parameters for an element type and precision
 * (us is ignored by vla_tune_set and 0 from vla_tune_get).  Errors:
 * VLA_ERR_INVALID_ARG for a NULL struct, an unknown element type or
 * precision, or (set) a budget outside [0, 65536] or residency outside
 * [0, 32]. */
vla_status vla_tune_get(int32_t dim, int32_t order, int32_t precision, vla_tune_t *out);
vla_status vla_tune_set(int32_t dim, int32_t order, int32_t precision, const vla_tune_t *in);

/* ------------------------------------------------------------------------ */
/* Assembly server: continuous batching over a device-memory budget          */
/* ------------------------------------------------------------------------ */
/* The paper has no server; this is the serving form of its assembly.  A
 * request carries a mesh (arrays plus a client key) and a coefficient and
 * returns K, M (in the mesh's CSR pattern) and vol, computed exactly as
 * vla_assemble computes them (bit-identical whatever else runs at the same
 * time).  Requests are admitted in arrival order while the memory they need
 * (the mesh handle, estimated until built, and the outputs) fits the budget;
 * idle resident meshes are evicted least recently used first to make room,
 * and a request that could never fit fails with VLA_ERR_BUDGET.  Ingest
 * threads build admitted meshes on their own streams while earlier requests
 * assemble; each scheduling step assembles every request whose mesh is ready
 * in ONE batched persistent launch, so requests that arrive while a launch
 * runs join the next one.  All calls are thread-safe. */

typedef struct vla_server vla_server;

typedef struct {
    int64_t hbm_budget_bytes;  /* device bytes the server may hold (meshes + outputs) */
    int32_t precision;         /* VLA_PREC_MIXED or VLA_PREC_FP64 for every request */
    int32_t ingest_workers;    /* host threads building meshes (0 = 4) */
    int32_t max_batch;         /* requests per launch at most (0 = no limit) */
    int32_t max_inflight;      /* admitted, unfinished requests at most (0 = no limit) */
} vla_server_config_t;

typedef struct {
    int64_t key;               /* >= 0: mesh identity; a request whose key names a mesh the
                                  server holds reuses it (the arrays are then not read).
                                  -1: a private mesh. */
    int32_t dim, order;
    int64_t nn, ne, nfb;
    const double *coords;      /* host or device; layouts as vla_mesh_create; read by the */
    const int32_t *elems;      /* ingest, so valid until the request is finished */
    const int32_t *faces;      /* or NULL (nfb 0) */
    int32_t keep_resident;     /* keep the mesh on the device under its key afterwards */
    int32_t coeff_kind;        /* as in vla_assemble */
    double ca, cb;
} vla_request_t;

typedef struct {
    int32_t status;            /* VLA_OK or the request's error */
    int32_t new_mesh;          /* 1 if this request built its mesh */
    int32_t batch_size;        /* requests in the launch that computed it */
    int32_t reserved;
    int64_t batch_id;
    int64_t nn, ne, nnz;
    const double *K_vals, *M_vals, *vol;   /* device; valid until vla_server_release */
    const int32_t *row_ptr, *col_idx;      /* device CSR pattern of the mesh; same lifetime */
    double t_submit, t_admit, t_ready, t_start, t_done;   /* CLOCK_MONOTONIC seconds */
    double t_ingest;           /* when an ingest thread took the request (0 if it reused a mesh) */
    double h2d_ms, build_ms;   /* device time of its input copy and of its mesh build (0 if reused) */
} vla_result_t;

typedef struct {
    int64_t budget_bytes, used_bytes, peak_bytes;
    int64_t n_done, n_failed, n_batches, n_ingested, n_reused, n_evicted, n_resident, n_queued, max_batch;
    double mean_batch;         /* requests per launch */
    double assembly_busy_s;    /* time with a launch in flight */
} vla_server_stats_t;

/* Starts the scheduler and ingest threads on the current device (serving of
 * the Section 3.5 assembly; no counterpart in the paper).  Errors:
 * VLA_ERR_INVALID_ARG for a NULL argument, a budget <= 0, an unknown
 * precision, ingest_workers outside [0, 64] or a negative limit; VLA_ERR_OOM;
 * VLA_ERR_CUDA if the streams cannot be created. */
vla_status vla_server_create(const vla_server_config_t *cfg, vla_server **out);

/* Queues a request (a mesh and a Section 3.5.1 coefficient); *ticket
 * identifies it.  Never blocks on the GPU.  Errors: VLA_ERR_INVALID_ARG for a
 * NULL argument, an unknown dim, order or coefficient kind, bad sizes or
 * arrays, or a server that is shutting down.  A request that fails later
 * (its mesh is invalid or can never fit the budget) reports its error
 * through vla_server_poll. */
vla_status vla_server_submit(vla_server *server, const vla_request_t *req, int64_t *ticket);

/* Serving (no counterpart in the paper): waits up to timeout_s seconds (0: no
 * wait) for the request: VLA_PENDING
 * while it runs, VLA_OK with *res filled when done, the request's error if
 * it failed (*res filled too).  Errors: VLA_ERR_INVALID_ARG for a NULL
 * server or an unknown ticket. */
vla_status vla_server_poll(vla_server *server, int64_t ticket, double timeout_s, vla_result_t *res);

/* Frees a finished request's outputs (and its mesh, unless resident); no
 * counterpart in the paper.  Errors: VLA_ERR_INVALID_ARG for a NULL server,
 * an unknown ticket or a request that has not finished. */
vla_status vla_server_release(vla_server *server, int64_t ticket);

/* Fills *stats (host struct): the server's counters (no counterpart in the
 * paper).  Errors: VLA_ERR_INVALID_ARG for a NULL argument. */
vla_status vla_server_stats(vla_server *server, vla_server_stats_t *stats);

/* Finishes admitted requests, drops queued ones, joins the threads and
 * frees everything (housekeeping; no counterpart in the paper).  NULL is a
 * no-op; cannot fail. */
vla_status vla_server_destroy(vla_server *server);

#ifdef __cplusplus
}
#endif

#endif /* VLA_H */
