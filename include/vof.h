/* vof.h — C ABI of the GB300 (sm_103a) sharp-interface VOF phase-change hot path.
 *
 * What the calls compute (paper: arXiv 2604.14938, Sec. 2.1 "Interface capturing method",
 * Eq. (edge_intersection) and the isoap steps; Sec. 2.3 "Energy specific terms", Eqs.
 * (mass_transfer), (front_interpolation), (extrapolation), (latent_source), (interface_htc);
 * Appendix B "Least Squares Gradient Reconstruction"):
 *
 *   vof_reconstruct          per interface cell (eps < alpha < 1 - eps): the vertex field
 *                            (inverse-distance average of alpha), the isovalue c whose liquid
 *                            sub-volume {phi >= c} equals alpha V, and the interface area A_int,
 *                            unit normal n_int (vapour -> liquid) and centroid x_gamma.
 *   vof_phase_change_source  interface-modified least-squares temperature gradient on the band
 *                            (interface cells and their face neighbours) with T_sat imposed at the
 *                            crossing point x_f of every face with (alpha_P-1/2)(alpha_Q-1/2) < 0;
 *                            per-side gradients; q_l = k_l (grad T_l . n) A_int,
 *                            q_v = -k_v (grad T_v . n) A_int; mdot = (q_l + q_v)/(h_lv V);
 *                            Q = -mdot h_lv; totals sum(mdot V), sum(Q V) by a fixed pairwise tree.
 *
 * The cut volume of a polyhedron is taken on its tetrahedralisation by its own vertices (faces
 * fanned from their lowest-id vertex, the cell fanned from its lowest-id vertex), phi linear per
 * tetrahedron: continuous and non-increasing in c, exact for linear fields.
 *
 * Conventions
 *   - Every function returns a vof_status; no exception or abort crosses the ABI. A non-zero
 *     status means malformed input, allocation failure or a CUDA error; vof_last_error() gives a
 *     thread-local message. Per-cell conditions (degenerate range, not converged, fallback,
 *     singular least squares, no neighbour on the other side) are status bits in arrays plus
 *     counters, never errors.
 *   - "stream" is a cudaStream_t passed as void*; all device work is ordered on it. Calls return
 *     without synchronising unless stated.
 *   - Device pointers are caller-owned unless stated; the library never frees them.
 *   - The mesh's faces must be planar (all generated meshes are) and its cells convex; at most
 *     VOF_MAX_CELL_VERTS vertices and VOF_MAX_CELL_TETS tetrahedra per cell.
 *   - Memory: vof_mesh_create allocates everything the mesh's steps need (geometry tables and a
 *     workspace sized for the mesh); the step calls allocate nothing.
 */
#ifndef VOF_H
#define VOF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VOF_MAX_CELL_VERTS 64
#define VOF_MAX_CELL_TETS 192

typedef enum {
  VOF_OK = 0,
  VOF_EINVAL = 1, /* bad argument (null pointer, size out of range, bad option) */
  VOF_ENOMEM = 2, /* device or host allocation failed */
  VOF_ECUDA = 3,  /* a CUDA call failed; see vof_last_error() */
  VOF_EMESH = 4,  /* malformed mesh (offsets, ids, face/cell lists disagree, cell too large) */
  VOF_ESTATE = 5  /* call out of order (e.g. source before reconstruct, no MLP loaded) */
} vof_status;

/* Per-cell status bits (int32 arrays). */
#define VOF_ST_DEGENERATE 1    /* phi_max - phi_min < 1e-14: c = phi_min, A_int = 0, mdot = 0 */
#define VOF_ST_NOT_CONVERGED 2 /* |V_L(c)/V - alpha| > tol after the iteration cap */
#define VOF_ST_FALLBACK 4      /* learned guess + secant missed tol; bracketed bisection finished it */
#define VOF_ST_SINGULAR_LSQ 8  /* det(G) <= 1e-12 (tr G / 3)^3: gradient set to 0 */
#define VOF_ST_NO_SIDE 16      /* no face neighbour looks into the other phase: its gradient is 0
                                * (options.extrap = 1: no counted inflow face, it keeps its own) */
#define VOF_ST_MLP_SKIPPED 32  /* more than 32 vertices: learned guess not used */

/* Crossing-point modes (Eq. front_interpolation). */
#define VOF_XF_RECON 0      /* x_f on the reconstructed interface plane (x_gamma, n_int) */
#define VOF_XF_LINEAR 1     /* x_f = x_o + t (x_n - x_o), t = (alpha_o - 1/2)/(alpha_o - alpha_n) */
#define VOF_XF_AS_PRINTED 2 /* t = |alpha_n - 1/2| / |alpha_o - alpha_n|, the equation as printed */

/* Root-search modes. */
#define VOF_ROOT_BISECT 0  /* plain FP64 bisection on [phi_min, phi_max] */
/* Learned: BF16 MLP guess refined on the FP32 pipe, then FP64: the cubic V_L of the vertex interval
 * that holds the refined point (one pass over the cell's tetrahedra), an evaluation at the refined
 * point, one at a Newton point, <= max_secant secant steps, bracketed bisection as the fallback.
 * Cells of at most 24 tetrahedra with one lane per cell (group_size 1, or the autotuner's choice)
 * take the thread-per-cell path instead (see root_narrow): the FP32 refinement stops once its
 * bracket holds no vertex value, the interval's cubic is summed in FP32 pairs, and safeguarded
 * Newton steps on it (up to 12) replace the Newton point and the secant steps. */
#define VOF_ROOT_LEARNED 1
/* Interval cubic: V_L(c) is one cubic between consecutive vertex values of a cell (Sec. 2.1 with
 * the cell split into tetrahedra of its own vertices); an FP32 refinement (from the MLP guess when
 * the mesh has an MLP, else from 1 - alpha) picks the interval, one
 * FP64 pass sums the straddling tetrahedra's pieces into that cubic, and its root follows from
 * the polynomial alone (bisection fallback, counted). The paper has no such mode. */
#define VOF_ROOT_CUBIC 2
/* Fixed isovalue: the iso-surface at alpha_iso (Sec. 2.1, typically 0.5), the paper's own
 * reconstruction, without volume matching; a cell whose vertex values do not straddle it has no
 * interface there. */
#define VOF_ROOT_FIXED 3

typedef struct vof_mesh vof_mesh; /* opaque, library-owned */

/* Mesh description: HOST pointers, read only during vof_mesh_create. Faces are vertex loops
 * oriented outward from their owner; cell_face entries have bit 31 set when the cell is the
 * face's neighbour (its loop is inward for that cell); face_neigh = -1 on the boundary. */
typedef struct {
  int64_t n_cells, n_faces, n_verts;
  const int64_t* cell_face_off; /* [n_cells + 1] */
  const int32_t* cell_face;     /* [cell_face_off[n_cells]] */
  const int64_t* face_vert_off; /* [n_faces + 1] */
  const int32_t* face_vert;     /* [face_vert_off[n_faces]] */
  const int32_t* face_owner;    /* [n_faces] */
  const int32_t* face_neigh;    /* [n_faces] */
  const double *vx, *vy, *vz;   /* [n_verts] */
} vof_mesh_desc;

typedef struct {
  double k_l, k_v; /* thermal conductivities of liquid and vapour, W/(m K) */
  double h_lv;     /* latent heat, J/kg */
  double T_sat;    /* saturation temperature, K */
} vof_props;

typedef struct {
  double alpha_eps;  /* interface cells: alpha_eps < alpha < 1 - alpha_eps (default 1e-12) */
  double tol_alpha;  /* root accepted when |V_L(c)/V - alpha| <= tol_alpha (default 1e-12) */
  int max_bisect;    /* bisection iteration cap (default 100) */
  int root_mode;     /* VOF_ROOT_BISECT, VOF_ROOT_LEARNED, VOF_ROOT_CUBIC or VOF_ROOT_FIXED */
  int max_secant;    /* secant steps after the learned guess (default 2; the lane-group path) */
  int xf_mode;       /* VOF_XF_* (default VOF_XF_RECON) */
  int vertex_mode;   /* 0 inverse distance to cell centroids (default), 1 plain average */
  int group_size;    /* lanes per cell in the root search: 0 = auto, else 1, 2, 4, 8, 16 or 32 */
  int htc;           /* 1: also compute the interface heat-transfer coefficients VOF_F_A_OWN and
                      * VOF_F_A_NEIGH (Eq. interface_htc) and each band cell's energy-matrix terms
                      * VOF_F_HTC_DIAG and VOF_F_HTC_RHS on a side branch of the step (default 0) */
  double alpha_iso;  /* isovalue of VOF_ROOT_FIXED, in (0, 1) (default 0.5) */
  /* Other-side gradient of an interface cell (Sec. 2.3, Eq. extrapolation):
   *   0 (default): one upwind sweep, the weighted mean of the gradients of the face neighbours on
   *     that side, weights max(0, +-n_int . A_f);
   *   1: the pseudo-time solve of Eq. (extrapolation), first-order upwind, one solve per side and
   *     gradient component. Unknowns: the interface cells of the other phase; every cell of the
   *     side keeps its modified least-squares gradient, which is also the unknowns' start value.
   *     The liquid side moves along -n_int, the vapour side along +n_int (from the bulk of the side
   *     towards the interface). Step dtau = min over faces of |d_f| (owner centroid to neighbour
   *     centroid, or to the face centroid on a boundary face: VOF_F_DTAU), limited per cell to
   *     V_P / sum of its inflow weights. A solve stops after the iteration whose largest change is
   *     below extrap_tol, or after extrap_max_iter; vof_counts.extrap_iters holds the counts.
   *     Needs cells of at most 64 faces (VOF_EINVAL otherwise). A batch is one mesh to the
   *     step: its dtau is the smallest over all its meshes, and a solve stops only when no mesh
   *     of the batch moves by extrap_tol or more. */
  int extrap;
  int extrap_max_iter; /* 1 .. 1000 (default 120) */
  double extrap_tol;   /* K/m, absolute, > 0 (default 1e-3) */
  /* Least-squares variants of the stencil-anisotropy study (Sec. 3, Fig. stencil_polar; Appendix B),
   * bits (default 0: the interface-modified face stencil, unweighted):
   *   1 the standard stencil: neighbours across the interface enter with their own centroid and
   *     temperature (no crossing point, no T_sat);
   *   2 inverse-distance weights w = 1/|r|^2 on every stencil entry (G = sum w r r^T, b = sum w r dT);
   *   4 the stencil of every cell sharing a vertex with the cell (boundary faces as before); in
   *     the modified stencil a neighbour across the interface that shares no face enters at the
   *     linear interpolation of alpha along the centroid connection, t = (a_P - 1/2)/(a_P - a_Q);
   *   8 also write cond(G_P) = lambda_max / lambda_min to VOF_F_LSQ_COND (band cells).
   * Any bit set runs the study's least-squares kernel (a thread per band cell) in place of the
   * path's; VOF_F_GRAD and everything downstream follow the chosen stencil. */
  int lsq_variant;
  /* Start of the FP32 refinement of VOF_ROOT_LEARNED and VOF_ROOT_CUBIC:
   *   0 (default): the MLP guess when the mesh has an MLP (VOF_ROOT_LEARNED requires one), else
   *     u0 = 1 - alpha;
   *   1: u0 = 1 - alpha for every cell, with or without an MLP: the learned path's refinement,
   *     FP64 window, secant steps and fallback without the network (no feature or MLP kernel
   *     runs), which measures what the network gains. */
  int guess;
  /* Reads of the pseudo-time extrapolation's per-iteration barrier word before a block stops
   * waiting (options.extrap = 1; default 4194304, range 1 .. 2^30). A block that stops waiting
   * ends the solve: every solve reports -1 iterations and the step's per-side gradients and
   * sources are invalid; the kernel returns normally and the next step is unaffected. */
  int extrap_poll_limit;
  /* Lanes per cell 1 (group_size, or the autotuner's choice) with VOF_ROOT_LEARNED or
   * VOF_ROOT_CUBIC, on cells of at most 24 tetrahedra, runs the thread-per-cell root search: its
   * root phase is in FP32-pair arithmetic (about 48 significant bits), with values normalised by
   * the cell's vertex range. A cell whose vertex interval around the root is narrower than
   * root_narrow times that range, or whose target no interval brackets, is handed to the FP64
   * lane-group path, which solves it from the start (default 2^-20, the narrowest interval the
   * pairs take; range 2^-20 .. 2; 2 hands every cell over). */
  double root_narrow;
} vof_options;

/* Fills *o with the defaults above. */
void vof_default_options(vof_options* o);

/* Builds a mesh: validates the arrays (VOF_EMESH on any inconsistency), derives the cell
 * tetrahedralisations, vertex->cell table and inverse-distance weights on the host, uploads
 * them, computes geometry (face area vectors and centroids, cell volumes and centroids,
 * tetrahedron volumes) on the device and allocates the step workspace. Synchronises the stream.
 * *out is library-owned; release it with vof_mesh_destroy. */
vof_status vof_mesh_create(const vof_mesh_desc* desc, void* stream, vof_mesh** out);
vof_status vof_mesh_destroy(vof_mesh* mesh);

/* Reconstruction. d_alpha: device [n_cells] liquid volume fractions. Results stay in the
 * mesh's workspace (see vof_copy_field). With VOF_ROOT_LEARNED an MLP must have been set with
 * vof_mlp_set_weights, else VOF_ESTATE. */
vof_status vof_reconstruct(vof_mesh* mesh, const double* d_alpha, const vof_options* opt, void* stream);

/* Phase-change source after vof_reconstruct with the same d_alpha. d_T: device [n_cells] cell
 * temperatures; d_T_bnd: device [n_faces] temperatures read at boundary faces (virtual
 * neighbours at the face centroid), or NULL to leave boundary faces out of the stencil.
 * d_mdot, d_Q: device [n_cells], written everywhere (zero outside interface cells).
 * d_totals: device [2] = {sum mdot V, sum Q V} over interface cells (pairwise tree in cell order). */
vof_status vof_phase_change_source(vof_mesh* mesh, const double* d_alpha, const double* d_T, const double* d_T_bnd,
                                   const vof_props* props, const vof_options* opt, double* d_mdot, double* d_Q,
                                   double* d_totals, void* stream);

/* One whole step: vof_reconstruct followed by vof_phase_change_source. */
vof_status vof_step(vof_mesh* mesh, const double* d_alpha, const double* d_T, const double* d_T_bnd,
                    const vof_props* props, const vof_options* opt, double* d_mdot, double* d_Q, double* d_totals,
                    void* stream);

/* The same step from HOST buffers: copies h_alpha, h_T [n_cells] (and the boundary entries of
 * h_T_bnd [n_faces] when non-NULL) to the device on the stream, runs vof_step, copies mdot
 * [n_cells] into h_mdot and the totals into h_totals [2], and synchronises. With every buffer in
 * pinned (mapped) host memory and a stream other than the default one, the boundary entries are
 * gathered through the mapping and the whole sequence is captured once into a CUDA graph and
 * replayed while the pointers, properties, options, tuned lanes and MLP stay the same; other
 * buffers take plain copies and eager launches. */
vof_status vof_step_host(vof_mesh* mesh, const double* h_alpha, const double* h_T, const double* h_T_bnd,
                         const vof_props* props, const vof_options* opt, double* h_mdot, double* h_totals,
                         void* stream);

/* vof_step replayed as a CUDA graph on a non-default stream: the first call, and any call whose
 * pointers, properties, options or tuned group sizes differ from the captured ones, captures
 * the whole step on the stream (relaxed capture mode) and instantiates it; other calls launch
 * the graph. Same arguments and results as vof_step. Kernel timing is not recorded inside it. */
vof_status vof_step_graph(vof_mesh* mesh, const double* d_alpha, const double* d_T, const double* d_T_bnd,
                          const vof_props* props, const vof_options* opt, double* d_mdot, double* d_Q, double* d_totals,
                          void* stream);

/* Interface cells are binned by tetrahedron count ([1,4], [5,8], [9,24], [25,64], [65,192]); each
 * bin's root search runs with its own lanes per cell G. vof_autotune reconstructs with d_alpha,
 * then, bin by bin (largest first), times reps whole reconstructions (CUDA events) for each of
 * G = 1, 2, 4, 8, 16, 32, the other bins at their current choice, and keeps the fastest;
 * synchronises; h_G_out [5] (may be NULL) gets the choice (0 for bins without interface cells).
 * The choice applies when opt->group_size is 0.
 * vof_set_group_sizes sets it directly (0 = the built-in default for that bin). A choice whose lane
 * groups do not fit in a block's shared memory in the step's root mode (plain bisection keeps FP64
 * rows, twice the other modes' bytes) runs with the next larger lane count that fits. */
vof_status vof_autotune(vof_mesh* mesh, const double* d_alpha, const vof_options* opt, int reps, int* h_G_out,
                        void* stream);
vof_status vof_set_group_sizes(vof_mesh* mesh, const int* h_G);

/* ---- batches of independent meshes (many meshes of uneven size and cell type in one launch)
 * ----
 * A batch is the disjoint union of n meshes: cells, faces and vertices renumbered with the offsets
 * vof_batch_offsets returns (host arrays of n + 1). vof_batch_mesh gives the union mesh, stepped
 * like any mesh (vof_step, vof_step_graph; alpha, T, T_bnd, mdot, Q concatenated in mesh order).
 * vof_batch_totals writes d_totals [n][2] = {sum mdot V, sum Q V} per mesh for the last step: the
 * pairwise tree over each mesh's interface cells, as a single-mesh step computes it (at most 4.2 M
 * interface cells per mesh). vof_batch_create synchronises. */
typedef struct vof_batch vof_batch;
vof_status vof_batch_create(const vof_mesh_desc* descs, int n_meshes, void* stream, vof_batch** out);
vof_status vof_batch_destroy(vof_batch* batch);
vof_status vof_batch_mesh(vof_batch* batch, vof_mesh** out);
vof_status vof_batch_offsets(const vof_batch* batch, int64_t* h_cells, int64_t* h_faces, int64_t* h_verts);
vof_status vof_batch_totals(vof_batch* batch, double* d_totals, void* stream);

/* Workspace fields, copied with vof_copy_field into caller device memory (count = elements). */
typedef enum {
  VOF_F_IFACE_IDX = 0, /* int32 [n_iface]: interface cells in increasing cell order */
  VOF_F_PHI_V = 1,     /* double [n_verts]: vertex field (valid on vertices of interface cells) */
  VOF_F_ISO = 2,       /* double [n_cells]: isovalue c (interface cells) */
  VOF_F_A_INT = 3,     /* double [n_cells] */
  VOF_F_N_INT = 4,     /* double [n_cells][3] */
  VOF_F_X_GAMMA = 5,   /* double [n_cells][3] */
  VOF_F_STATUS = 6,    /* int32 [n_cells]: VOF_ST_* bits (interface and band cells) */
  VOF_F_EVALS = 7,     /* int32 [n_cells]: FP64 cut-volume evaluations of the root search: passes over the
                        * cell's tetrahedra (a bisection evaluation, or the cubic of a vertex interval on
                        * the learned and interval-cubic paths, whose evaluations at points of the
                        * interval are then scalar) */
  VOF_F_GRAD = 8,      /* double [n_cells][3]: modified least-squares grad T (band cells) */
  VOF_F_GRAD_L = 9,    /* double [n_cells][3]: liquid-side gradient (interface cells) */
  VOF_F_GRAD_V = 10,   /* double [n_cells][3]: vapour-side gradient (interface cells) */
  VOF_F_Q_L = 11,      /* double [n_cells] */
  VOF_F_Q_V = 12,      /* double [n_cells] */
  VOF_F_X_F = 13,      /* double [n_faces][3]: crossing point (crossing faces next to the band) */
  VOF_F_D_OWN = 14,    /* double [n_faces]: |x_f - x_owner| */
  VOF_F_D_NEIGH = 15,  /* double [n_faces]: |x_f - x_neigh| */
  VOF_F_A_INT_F = 16,  /* double [n_faces]: |A_int n_int . n_f| of the interface cell used */
  VOF_F_FACE_STAMP = 17, /* uint32 [n_faces]: equals the step stamp on crossing faces of this step */
  VOF_F_CELL_VOL = 18, /* double [n_cells] */
  VOF_F_CELL_CEN = 19, /* double [n_cells][3] */
  VOF_F_FACE_AREA = 20,/* double [n_faces][3], outward from the owner */
  VOF_F_FACE_CEN = 21, /* double [n_faces][3] */
  VOF_F_IFACE_STAMP = 22, /* uint32 [n_cells]: equals the step stamp on interface cells */
  VOF_F_BAND_STAMP = 23,  /* uint32 [n_cells]: equals the step stamp on band cells */
  VOF_F_A_OWN = 24,    /* double [n_faces]: a_f = k_phi A_int,f / d_own of the owner side (Eq. interface_htc) */
  VOF_F_A_NEIGH = 25,  /* double [n_faces]: the same for the neighbour side; both on crossing faces next to
                        * the band, in steps run with options.htc = 1: each side adds a_f to its
                        * energy-matrix diagonal and a_f T_sat to its right-hand side, the face being
                        * detached from the diffusive coupling (per-cell sums: VOF_F_HTC_DIAG/RHS) */
  VOF_F_DTAU = 26,     /* double [1]: pseudo-time step of Eq. (extrapolation), min over faces of |d_f| */
  VOF_F_LSQ_COND = 27, /* double [n_cells]: cond(G_P) of band cells, in steps run with options.lsq_variant bit 8
                        * (inf where G_P has no positive smallest eigenvalue) */
  /* Energy-matrix terms of Eq. interface_htc (Sec. 2.3, heat source/sink), in steps run with
   * options.htc = 1, valid on band cells (VOF_F_BAND_STAMP): per cell, over its faces detached by the
   * interface (the crossing faces of the step) in the cell's face order, the sum of its own side's
   * a_f (added to the cell's diagonal) and the sum of a_f T_sat (added to its right-hand side).
   * No cell outside the band has such a face with a non-zero coefficient. */
  VOF_F_HTC_DIAG = 28, /* double [n_cells] */
  VOF_F_HTC_RHS = 29,  /* double [n_cells] */
  VOF_F_N = 30
} vof_field;

/* Element count of a field in the current state (n_iface for the interface list). */
vof_status vof_field_size(vof_mesh* mesh, int field, int64_t* count, int* elem_bytes);
/* Copies a field into d_dst (device, at least count * elem_bytes bytes) on the stream; d_dst may be
 * NULL when count is 0. */
vof_status vof_copy_field(vof_mesh* mesh, int field, void* d_dst, int64_t count, void* stream);

/* Counters of the last step, read back synchronously. */
typedef struct {
  int64_t step;  /* stamp of the last step (see the *_STAMP fields) */
  int64_t n_iface, n_band, n_crossing;
  int64_t n_degenerate, n_not_converged, n_fallback, n_singular, n_no_side, n_mlp_skipped;
  int64_t evals_total; /* FP64 cut-volume evaluations (VOF_F_EVALS) summed over interface cells */
  /* algorithmic work of the root search (roofline accounting): tetrahedron evaluations (sum over
   * interface cells of evaluations x tetrahedra), tetrahedra prepared, tetrahedra cut by the final
   * interface */
  int64_t tet_evals, tets_prepared, tets_sectioned;
  int64_t evals32_total; /* FP32 evaluations of the learned path's refinement */
  /* iterations of the six pseudo-time solves of options.extrap = 1 (liquid side x, y, z, then
   * vapour side x, y, z); 0 in steps with options.extrap = 0; -1 for every solve when a block of the
   * launch gave up waiting at the iteration barrier (a bounded poll; the step's per-side
   * gradients and sources are then invalid) */
  int64_t extrap_iters[6];
} vof_counts;
vof_status vof_get_counts(vof_mesh* mesh, vof_counts* out, void* stream);

/* Mesh sizes and limits: n_cells, n_faces, n_verts, max vertices per cell, max tets per cell. */
vof_status vof_mesh_info(const vof_mesh* mesh, int64_t* out5);

/* Cells of the mesh per tetrahedron-count bin (1-4, 5-8, 9-24, 25-64, 65-192 tetrahedra):
 * a step launches the root search once for every non-empty bin (then the interface geometry
 * once over all interface cells).
 * Host array of 5.
 * No counterpart in the paper (launch layout of this implementation). */
vof_status vof_mesh_bins(const vof_mesh* mesh, int64_t* cells5);

/* ---- learned isovalue guess (the learned part of the path; the paper fixes no such model) ----
 * A 40 -> 64 -> 64 -> 64 -> 1 GELU MLP predicting the normalised isovalue position
 * t = (c - phi_min)/(phi_max - phi_min) of an interface cell. BF16 operands with FP32
 * accumulation (forward and backward on the tensor cores), FP32 master weights and Adam.
 * Parameters (float32, row-major): W1[64][40], b1[64], W2[64][64], b2[64], W3[64][64], b3[64],
 * w4[64], b4. Features (float32 [n][40]): alpha; faces/32; the vertex values normalised to [0,1]
 * over the cell's range, sorted descending, padded to 32 with the smallest; bounding-box extents
 * / V^(1/3) (3); (vertex mean - bounding-box centre) / V^(1/3) (3). Cells with more than 32
 * vertices or a degenerate range have no features (VOF_ST_MLP_SKIPPED: plain bisection). */
#define VOF_MLP_N_PARAMS 11009
#define VOF_MLP_N_FEATURES 40
#define VOF_MLP_MAX_BATCH 65536
typedef struct vof_mlp vof_mlp; /* opaque, library-owned, device memory allocated at creation */

/* Creates an MLP from host parameters (VOF_MLP_N_PARAMS floats); synchronises the device. */
vof_status vof_mlp_create(const float* h_params, vof_mlp** out);
vof_status vof_mlp_destroy(vof_mlp* mlp);
/* Copies the FP32 master parameters to the host; synchronises. */
vof_status vof_mlp_get_params(vof_mlp* mlp, float* h_params);
/* d_y[i] = MLP(d_X[i]) for i < n (device float32, features [n][40]). */
vof_status vof_mlp_forward(vof_mlp* mlp, const float* d_X, int64_t n, float* d_y, void* stream);
/* One Adam step (beta 0.9, 0.999, eps 1e-8) on the mean squared error of a batch of
 * n <= VOF_MLP_MAX_BATCH samples (d_t [n] targets); d_loss (device float [1], may be NULL) gets
 * the batch loss before the step. Gradient partials are summed in a fixed order. */
vof_status vof_mlp_train_step(vof_mlp* mlp, const float* d_X, const float* d_t, int64_t n, float lr, float* d_loss,
                              void* stream);
/* The gradient of the batch loss (device float [VOF_MLP_N_PARAMS]) without an update. */
vof_status vof_mlp_grad(vof_mlp* mlp, const float* d_X, const float* d_t, int64_t n, float* d_grad, float* d_loss,
                        void* stream);
/* Attaches an MLP (or NULL) to a mesh for VOF_ROOT_LEARNED; on first use allocates the mesh's
 * feature buffers and computes every cell's mesh-only features (faces / 32 and the six shape
 * features) once, synchronising the device. The MLP must outlive its use by the mesh. */
vof_status vof_mesh_set_mlp(vof_mesh* mesh, vof_mlp* mlp);
/* Features of the interface cells of the last reconstruction, made with that reconstruction's
 * d_alpha: d_X [n_iface][40], d_ok [n_iface] (1 where the cell has features). On a mesh without an
 * MLP attached, the first call allocates the buffer of the mesh-only features and fills it. */
vof_status vof_mlp_features(vof_mesh* mesh, const double* d_alpha, float* d_X, int32_t* d_ok, void* stream);

/* ---- totals without allocation (no counterpart in the paper: a variant of the totals step) ----
 * Some callers cannot allocate device memory where they need the totals: code that runs while
 * its stream is being captured into a CUDA graph, real-time loops that must not enter an
 * allocator, hosts that hand out all device memory from their own pool. vof_totals_static
 * computes the same pairwise-tree sums as the d_totals of vof_phase_change_source,
 * d_totals[0] = sum d_a[i], d_totals[1] = sum d_b[i] (i < n, zero-padded to a power of two, pairs
 * summed level by level), over caller-supplied device arrays (e.g. mdot V and Q V of the interface
 * cells in cell order). It allocates nothing: its chunk sums live in a 32 KB file-scope device
 * array that every GPU loading the library holds until exit. The first call made with a device
 * current looks up that array's address (cudaGetSymbolAddress); make that first call before any
 * stream capture. The address is kept per device for the life of the process: do not call the
 * function on a device after cudaDeviceReset on it (the kept address would be stale). Every call shares the array and zeroes its block counter before launching, so
 * calls that overlap on the GPU (two streams, or two host threads) race; order them on one stream.
 * n > VOF_TOTALS_STATIC_MAX_N returns VOF_EINVAL. */
#define VOF_TOTALS_STATIC_MAX_N 4194304
vof_status vof_totals_static(const double* d_a, const double* d_b, int64_t n, double* d_totals, void* stream);

/* Per-kernel device time, measured with pairs of CUDA events recorded on the launch stream
 * around each kernel group (off by default; measurement support, not part of the method).
 * vof_timing_enable(mesh, 1) creates the events on first use and resets the record;
 * vof_timing_read synchronises the stream and returns, per kernel class, the summed
 * milliseconds and the launch count since the last read (at most 8192 records are kept).
 * Classes, one per kernel: 0 selection, band and vertex field; 1 features of the learned guess;
 * 2 root search (one launch per non-empty bin, on parallel branches: their times add up);
 * 3 list of the crossing faces (a side branch in vof_step); 4 crossing points; 5 least squares;
 * 6 MLP forward pass of the learned guess; 7 interface geometry; 8 pseudo-time extrapolation
 * (options.extrap = 1); 9 per-side gradients, source and totals; 10 heat-transfer coefficients
 * (options.htc = 1, a side branch). */
vof_status vof_timing_enable(vof_mesh* mesh, int on);
vof_status vof_timing_read(vof_mesh* mesh, double* ms, int64_t* launches, int n, void* stream);

/* FP64 FMA throughput of the current device, the denominator of the roofline of the FP64-bound
 * kernels (measurement support; the paper has no counterpart). Launches a kernel whose threads
 * each run 8 independent FMA chains of `iters` steps, every SM at full occupancy: one untimed
 * launch, then `reps` launches timed with CUDA events on the stream. *h_ms = the fastest launch,
 * *h_flops = its FP64 flops (2 per FMA). Allocates a small output buffer for the launch's lifetime
 * and synchronises; iters < 1 or reps < 1 returns VOF_EINVAL. */
vof_status vof_probe_fp64_fma(int64_t iters, int reps, double* h_ms, double* h_flops, void* stream);

const char* vof_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* VOF_H */
