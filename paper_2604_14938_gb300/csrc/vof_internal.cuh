// Library-internal declarations shared by the CUDA sources of libvof_gb300.so.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "vof.h"

namespace vof {

// Order-preserving map of a double onto uint64 (-0.0 folded onto +0.0) and its inverse: integer
// operations only, so that comparisons, minima and maxima of FP64 values stay off the FP64 pipe.
__device__ __forceinline__ uint64_t okey(double x) {
  uint64_t b = (uint64_t)__double_as_longlong(x);
  b = b == 0x8000000000000000ull ? 0ull : b;
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double okey_inv(uint64_t k) {
  const uint64_t b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
  return __longlong_as_double((long long)b);
}

// Device counters of one step; reset by the step's first kernel.
struct Counters {
  uint32_t step;        // incremented on the device every step (membership stamps)
  uint32_t reduce_done; // blocks finished in the totals reduction
  int64_t n_iface, n_band, n_crossing;
  int64_t n_uvert;  // distinct vertices of interface cells (vertex field values computed)
  int64_t n_degenerate, n_not_converged, n_fallback, n_singular, n_no_side, n_mlp_skipped;
  int64_t evals_total;
  // algorithmic work of the root search: tetrahedron evaluations (sum of evals x tets per cell),
  // tetrahedra prepared, tetrahedra cut in the final geometry
  int64_t tet_evals, tets_prepared, tets_sectioned;
  int64_t evals32_total;  // FP32 evaluations of the learned path's refinement
  int64_t bin_count[5];   // interface cells per tetrahedron-count bin
  int64_t bin_next[5];    // next bin-list position to take (cells fetched dynamically by the root search)
  int64_t slow_count[5];  // cells the thread-per-cell root search hands to the lane-group kernel, per bin
  int64_t slow_next[5];   // next slow-list position to take
  int64_t extrap_iters[6];  // iterations of the pseudo-time solves (liquid x, y, z, vapour x, y, z)
};

// Everything a step kernel reads or writes, by value (device pointers).
struct MeshView {
  int64_t n_cells, n_faces, n_verts;
  const int64_t* cell_face_off;
  const int32_t* cell_face;
  const int32_t* face_owner;
  const int32_t* face_neigh;
  const double *vx, *vy, *vz;
  const int64_t* cell_vert_off;
  const int32_t* cell_vert;  // sorted unique vertex ids per cell; local 0 is the apex
  const int64_t* cell_tet_off;
  const uint32_t* cell_tet;  // three local vertex indices (8 bits each) of the base triangle
  const double* tet_vol;     // positive volumes, apex = local vertex 0
  const float* tet_vfrac;    // tet_vol / cell volume, FP32
  const float2* rel_pos;     // [cell-vertex entry][3]: vertex - apex of the cell, as (hi, lo) float pairs
  const int64_t* vert_cell_off;
  const int32_t* vert_cell;
  const double* vert_w;      // inverse-distance weights, normalised per vertex
  const double* cell_vol;
  const double* cell_ivol;   // 1 / cell_vol
  const double* cell_cen;    // [n][3]
  const double* face_area;   // [n][3] outward from owner
  const double* face_cen;    // [n][3]
  const double* face_len;    // [n] |x_neigh - x_owner| (0 on boundary faces)
  const double* face_iarea;  // [n] 1 / |face_area|
};

struct Workspace {
  Counters* counters;
  int32_t* iface_idx;      // [n_cells]
  int32_t* iface_slot;     // [n_cells] position of an interface cell in iface_idx (valid on this step's)
  uint32_t* iface_stamp;   // [n_cells]
  uint32_t* band_stamp;    // [n_cells]
  uint32_t* vert_stamp;    // [n_verts]
  uint32_t* face_stamp;    // [n_faces]
  uint32_t* sel_mask;      // [n_sel_blocks][kSelTile / 32] interface flags of the selection tiles
  int64_t* sel_tot;        // [kMaxSelGrid] interface cells per selection block
  int32_t* band_idx;       // [n_cells] band cells (unordered)
  double* phi_v;           // [n_verts]
  float2* phi_ff;          // [n_verts] phi_v as a (hi, lo) float pair
  double* iso;             // [n_cells]
  double* A_int;           // [n_cells]
  double* n_int;           // [n_cells][3]
  double* x_gamma;         // [n_cells][3]
  int32_t* status;         // [n_cells]
  int32_t* evals;          // [n_cells]
  double* grad;            // [n_cells][3]
  double* grad_l;          // [n_cells][3]
  double* grad_v;          // [n_cells][3]
  double* q_l;             // [n_cells]
  double* q_v;             // [n_cells]
  double* x_f;             // [n_faces][3]
  double* d_own;           // [n_faces]
  double* d_neigh;         // [n_faces]
  double* A_int_f;         // [n_faces]
  double *a_own, *a_neigh;  // [n_faces]: interface heat-transfer coefficients of the two sides
  double *htc_diag, *htc_rhs;  // [n_cells]: sum of a_f, sum of a_f T_sat over a band cell's detached faces
  int32_t* xface_list;     // [n_faces] crossing faces next to the band (n_crossing of them this step)
  double* mdotV;           // [n_cells] in interface-list order
  double* QV;              // [n_cells]
  double* partial;         // [4][kMaxPartials]: two ping-pong buffers per total
  double* tile_part;       // [2][ceil(n_cells / kSrcTile)]: totals of aligned tiles of the interface list
  float* mlp_out;          // [n_cells] learned guesses (normalised position in the range)
  int32_t* bin_list;       // [kBins][n_cells] interface-list positions per bin
  int32_t* slow_list;      // [kBins][n_cells] bin-list entries left to the lane-group root search
  const double* alpha_in;  // alpha of the current step
  float* mlp_x;            // [n_cells][40] features of interface cells (allocated with an MLP)
  int32_t* mlp_ok;         // [n_cells] 1 where the cell has features
  float* mlp_y;            // [n_cells] raw MLP outputs
  float* mlp_static;       // [n_cells][8] faces / 32 and the six shape features (allocated with an MLP)
  // pseudo-time extrapolation (options.extrap = 1), per interface-list slot
  double* ex_x;            // [2][n_cells][4] iterates of the slot's other-side gradient (ping-pong, padded)
  double* ex_k;            // [n_cells][5]: C = sum of step weights, f = dtau_P / V_P, b (3) = known inflow
  int32_t* ex_nb;          // [n_cells][kExCap] slots of the first unknown neighbours (-1: none)
  double* ex_g;            // [n_cells][kExCap] their step weights f_P w_f
  unsigned long long* ex_mask;  // [n_cells] face positions of further unknown neighbours
  unsigned long long* ex_itmax; // [kExMaxIter + 1] per iteration: barrier word (arrivals, blocks still moving)
  double* ex_dtau;         // [1] min over faces of |d_f|
  double* lsq_cond;        // [n_cells] cond(G_P) of band cells (least-squares study variants)
  // device staging for the host-buffer step
  double *io_alpha, *io_T, *io_Tb, *io_mdot, *io_Q, *io_totals;
};

constexpr int kSelTile = 512;       // cells per selection tile (2 consecutive cells per thread)
constexpr int kMaxSelGrid = 4096;   // blocks of the cooperative selection launch, at most
// Bins of interface cells by tetrahedron count; each bin's root search has its own lanes per cell.
constexpr int kBins = 5;
constexpr int kBinMaxTets[kBins] = {4, 8, 24, 64, 192};
__host__ __device__ inline int bin_of(int nt) { return nt <= 4 ? 0 : (nt <= 8 ? 1 : (nt <= 24 ? 2 : (nt <= 64 ? 3 : 4))); }
constexpr int kReduceChunk = 2048;  // leaves per reduction block (power of two)
constexpr int kSrcTile = 256;       // interface cells per source tile (an aligned subtree of the totals)
constexpr int kMaxPartials = 8192;  // reduction blocks (n_iface <= 16.7 M)
constexpr int kExMaxIter = 1000;    // cap of options.extrap_max_iter
constexpr int kExMaxFaces = 64;     // faces per cell the extrapolation's face masks cover
constexpr int kExCap = 8;           // unknown neighbours per slot gathered once (the rest: face mask)

struct StepArgs {
  const double* alpha;
  const double* T;
  const double* T_bnd;
  double* mdot;
  double* Q;
  double* totals;
  vof_props props;
  vof_options opt;
};

}  // namespace vof

namespace vof {
// Optional per-kernel device timing: pairs of CUDA events recorded on the launch stream.
// one class per kernel of the step (the root search: one launch per non-empty bin)
enum KernelClass {
  KC_SELECT = 0, KC_MLP_FEATURES, KC_ROOT, KC_XMARK, KC_XFACE, KC_LSQ, KC_MLP_FORWARD, KC_GEOM, KC_EXTRAP,
  KC_SOURCE, KC_HTC, KC_N
};
struct Timing {
  bool on = false;
  int cap = 0, used = 0;
  std::vector<cudaEvent_t> ev;  // 2 per record
  std::vector<int> cls;
  void start(int k, cudaStream_t s) {
    if (!on || used >= cap) return;
    cls[used] = k;
    cudaEventRecord(ev[2 * used], s);
  }
  void stop(cudaStream_t s) {
    if (!on || used >= cap) return;
    cudaEventRecord(ev[2 * used + 1], s);
    ++used;
  }
};
}  // namespace vof

namespace vof {
// A captured step: the graph is valid while the arguments it bakes in (the key) are unchanged.
struct GraphCache {
  cudaGraphExec_t exec = nullptr;
  std::vector<unsigned char> key;
  int64_t captures = 0;
};
}  // namespace vof

struct vof_mesh {
  int64_t n_cells = 0, n_faces = 0, n_verts = 0;
  int max_cv = 0, max_ct = 0, max_cf = 0;  // vertices, tetrahedra, faces of the largest cell
  double mean_ct = 0;  // tetrahedra per cell, mean
  int64_t bin_cells[vof::kBins] = {0, 0, 0, 0, 0};  // cells of the mesh per bin
  int bin_max_ct[vof::kBins] = {0, 0, 0, 0, 0};     // largest tetrahedron count per bin
  int bin_G[vof::kBins] = {0, 0, 0, 0, 0};          // lanes per cell (autotuned; 0 = default)
  int n_sel_blocks = 0;
  int num_sms = 0;
  int sel_grid = 0;   // blocks of the cooperative selection launch (all resident)
  int geom_grid = 0;  // blocks of the interface-geometry launch
  int geom_bmax = 0;  // interface cells per warp batch of the geometry
  int ex_grid = 0;    // blocks of the cooperative extrapolation launch
  int32_t* bnd_faces = nullptr;  // device list of the boundary faces (face_neigh < 0)
  int64_t n_bnd = 0;
  vof::MeshView view{};
  vof::Workspace ws{};
  std::vector<void*> allocs;
  // learned isovalue guess (BF16 weights, device), see vof_mlp.cu
  vof_mlp* mlp = nullptr;
  bool recon_done = false;
  vof::Timing timing;
  vof::GraphCache graph;       // vof_step_graph
  vof::GraphCache host_graph;  // vof_step_host with pinned buffers
  // the bins' root searches run as parallel branches (fork after binning, join before the
  // interface geometry), so that one bin's slow cells overlap the other bins' work
  cudaStream_t bin_stream[vof::kBins] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_join[vof::kBins] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  // side branch of a whole step: crossing-face list, from the band to the least squares
  cudaStream_t xm_stream = nullptr;
  cudaEvent_t ev_xfork = nullptr, ev_xjoin = nullptr;
  // zeros of mdot and Q (every cell; the source then writes the interface cells): a memset on
  // its own branch, forked when the source stage starts and joined before the source kernel
  cudaStream_t z_stream = nullptr;
  cudaEvent_t ev_zfork = nullptr, ev_zjoin = nullptr;
  // host-buffer step: T and T_bnd are copied on their own stream while the reconstruction runs;
  // the source stage waits for ev_io_done when io_pending is set
  cudaStream_t io_stream = nullptr;
  cudaEvent_t ev_io_start = nullptr, ev_io_done = nullptr;
  bool io_pending = false;
};

namespace vof {
void set_error(const std::string& msg);
vof_status cuda_fail(cudaError_t e, const char* what);

// step kernels (vof_step.cu)
// early_xmark: the step's source stage will use the same alpha, so the crossing faces are listed
// on a side branch as soon as the band is known, and launch_source(..., xmark_done = true) only
// joins that branch.
vof_status launch_reconstruct(vof_mesh* m, const double* d_alpha, const vof_options& opt, cudaStream_t s,
                              bool early_xmark = false);
vof_status launch_source(vof_mesh* m, const StepArgs& a, cudaStream_t s, bool xmark_done = false);
cudaError_t launch_root_bin(vof_mesh* m, const double* alpha, const vof_options& opt, cudaStream_t s, int learned,
                            int bin, int G);
}  // namespace vof
