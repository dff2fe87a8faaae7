// plan.cuh -- the plan object behind fmm_plan_t: tree, lists, operators and
// evaluation workspace, all resident in HBM.
#pragma once
#include "common.cuh"

namespace fmm {

struct M2LTile {
  int32_t start;   // first entry in m2l_order
  int32_t count;   // targets in this tile (<= tile size)
  int32_t parity;  // octant parity shared by the tile's targets (bit0 x, bit1 y, bit2 z)
  int32_t pad;
};

struct Operators {
  int order = -1;
  // scale-free real-basis matrices, row-major [out][in], NC = (p+1)^2:
  //   m2l[343][NC][NC] indexed by offset code (dx+3)*49+(dy+3)*7+(dz+3),
  //   d = anchor(target) - anchor(source); m2m[8], l2l[8] by child octant.
  DBuf<double> m2l64, m2m64, l2l64;
  DBuf<float> m2l32, m2m32, l2l32;
  // FP32 M2M / L2L, input-major with the outputs contiguous and zero padded:
  // [8][(p+1)^2][coef_pitch(p)] (4 outputs per 16-byte load)
  DBuf<float> m2m32t, l2l32t;
  // FP32 M2L, output-major and zero padded: m2l32p[343][m2l_rows(p)][coef_pitch(p)]
  DBuf<float> m2l32p;
  // tensor-core M2L: TF32 hi/lo halves in the MMA's core-matrix order, and
  // the FP16 form (hi/lo halves of the balanced operators, their row and
  // column power-of-two scales)
  DBuf<float> m2l_tc;
  DBuf<uint16_t> m2l_tc16;
  DBuf<float> m2l_tc16_rows, m2l_tc16_cols;
  // rotated M2L (built when a plan uses it): per offset code, the real
  // block-diagonal rotation taking the offset to the z axis, applied to the
  // multipole (rot[code][0]) and back to the local (rot[code][1]), each
  // sum_n (2n+1)^2 entries, block n at n(2n-1)(2n+1)/3, row-major [out][in];
  // and the z-axis translation zt[code][n][k] = (n+k)! / |d|^(n+k+1)
  int rot_order = -1;
  DBuf<double> rot64, zt64;
  DBuf<float> rot32, zt32;
};

// Helmholtz mat-vec (helmholtz.cu): translation operators for one (kappa,
// order, root cube, depth) -- per level, input-major [k][j] complex --, and the
// evaluation workspace (multipoles, locals, sorted charges, far field)
struct HelmholtzState {
  double kappa = 0.0, D = 0.0;
  int order = -1, nlevels = 0;
  bool f32 = false;  // mixed plans: the M2L operators also in scaled FP32 (m2l32)
  DBuf<double> gaunt;
  DBuf<double2> m2l, m2m, l2l, xtab;
  DBuf<float2> m2l32;
  DBuf<double2> M, L, q, far;
};

// passes timed by the optional profiler (fmm_profile / fmm_profile_read)
enum Pass { kPassSort = 0, kPassBoxes, kPassLists, kPassP2M, kPassM2M, kPassM2L, kPassP2L,
            kPassL2L, kPassL2P, kPassM2P, kPassP2P, kPassReduce, kNumPasses };

uint64_t launch_count();

struct fmm_plan_impl {
  // configuration
  int m2l_path = 0;                  // 0 auto, 1 CUDA cores, 2 tensor cores, 3 rotated
  bool m2l_rot = false;              // this plan's M2L uses the rotated operators
  bool dual = false;                 // lists from the dual-tree walk (else U/V/W/X)
  double theta = 0.5;                // dual tree: acceptance r_T + r_S < theta |c_T - c_S|
  bool m2l_tc = false;               // this plan's M2L runs on the tensor cores
  int m2l_tile = 0;                  // tensor-core form: 0 default, 1 TF32 split, 2 FP16 split
  int order = 0, leaf_size = 1, autotune = 0, precision = FMM_FP64, coarse_fp64_levels = 3, max_depth = kMaxDepth;
  // W pairs of two leaves whose W leaf holds at most this many points go to
  // the near field in both directions (0 = off; opts.wx_direct sets (p+1)^2)
  int wx_direct_max = 0;
  cudaStream_t stream = nullptr;
  // host-buffer calls: a side stream for copies that overlap the computation,
  // and the events that order it against `stream` (created on first use)
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t copy_ev[4] = {nullptr, nullptr, nullptr, nullptr};

  // problems: a plan holds one problem, or a batch of independent problems
  // (a forest: each problem has its own root cube and tree; they never
  // interact).  Problem b owns input points [prob_off_h[b], prob_off_h[b+1]).
  int nproblems = 1;
  std::vector<int64_t> prob_off_h;
  DBuf<int64_t> prob_off;
  DBuf<double> prob_geom;           // per problem: lo[3], D, non-finite flag, pad
  std::vector<double> prob_geom_h;

  // points
  int64_t n = 0;
  double lo[3] = {0, 0, 0}, D = 1.0;
  DBuf<double> geom;                // device: lo[3], D, nonfinite flag
  DBuf<double> partial;             // bbox partials
  DBuf<uint64_t> keys, keys_tmp;    // sorted Morton keys
  DBuf<int32_t> perm, perm_tmp;     // sorted position -> input index
  DBuf<int32_t> iperm;              // input index -> sorted position
  DBuf<double> xyz_sorted;          // n x 3 (sorted order)
  DBuf<Dbl4> pl64;               // per sorted point: position - leaf centre (w unused)
  DBuf<float4> pl32;                // FP32 copy of pl64

  // boxes, numbered by (level, key)
  int nlevels = 0;
  std::vector<int32_t> level_off;   // host, nlevels + 1
  int64_t nboxes = 0;
  DBuf<uint64_t> box_key;
  DBuf<int32_t> box_level, box_first, box_count, box_parent, box_child, box_nchild;
  DBuf<BoxGeo> box_geo;
  DBuf<int32_t> box_prob;           // problem of each box
  DBuf<double> box_side;            // side length of each box
  DBuf<int32_t> colleagues;         // nboxes x 26, sorted, -1 padded
  DBuf<int32_t> ncolleagues;

  // lists (CSR over all boxes); a dual-tree plan keeps its P2P leaf pairs in
  // U and its M2L pairs (sources of any level) in V, with W and X empty
  DBuf<int32_t> u_off, u_idx, v_off, v_idx, w_off, w_idx, x_off, x_idx;
  DBuf<double> radius;              // dual tree: max |x_j - c_B| over the box's points
  DBuf<int2> dt_a, dt_b, dt_m2l, dt_p2p;  // dual-tree walk: frontiers and pairs
  DBuf<unsigned long long> dt_cnt;
  // dual tree, mixed precision: the M2L pairs split into those of the tensor-core
  // tiles (same level, offset in the operator table) and the rest
  DBuf<int32_t> dt_toff, dt_tidx, dt_goff, dt_gidx;
  int64_t ndt_t = 0, ndt_g = 0;
  int64_t nu = 0, nv = 0, nw = 0, nx = 0;
  bool v_built = true;              // false: V is built on request (build_vlists)

  // work lists
  DBuf<int32_t> leaves;             // leaf boxes
  int64_t nleaves = 0;
  DBuf<int32_t> xboxes;             // boxes with a non-empty X list (= the W sources)
  int64_t nxboxes = 0;
  DBuf<int32_t> xslot;              // per box: its index in xboxes, or -1
  DBuf<int32_t> wleaves;            // leaves with a non-empty W list
  int64_t nwleaves = 0;
  DBuf<int32_t> m2l_order;          // boxes of level >= 2 ordered by (level, parity, index)
  DBuf<M2LTile> m2l_tiles;
  int64_t nm2l_tiles = 0;
  int m2l_tile_size = 0;
  // per tile: source box of every (slot, target) (-1 = none), and the
  // occupied slots in ascending order
  DBuf<int32_t> m2l_src;            // ntiles x 216 x tile
  DBuf<int16_t> m2l_slots;          // ntiles x 216
  DBuf<int32_t> m2l_nslots;         // ntiles

  // operators (rebuilt only when the order changes)
  Operators ops;

  // evaluation workspace
  DBuf<Dbl4> src64;              // per sorted point: (local x, y, z, q)
  DBuf<float4> src32;
  DBuf<float> p2p_pairs;            // FP32 near field: every leaf's sources packed in pairs
  DBuf<int4> p2p_meta;              // FP32 near field: staging record per U entry
  DBuf<float> p2p_meta_z;
  DBuf<uint64_t> p2p_key, p2p_key_tmp;
  DBuf<int32_t> p2p_order, p2p_order_tmp;  // leaves, most near-field work first
  DBuf<int32_t> p2p_ticket;
  bool p2p_meta_ok = false;         // p2p_meta and p2p_order match the current lists
  // FP32 M2M / L2L: the boxes of each level grouped by octant within the
  // parent (oct_order), group l * 9 + o starting at oct_off[l * 9 + o]
  // (oct_off[l * 9 + 8] = end of level l); oct_pos is scratch
  DBuf<int32_t> oct_off, oct_order, oct_pos;
  bool oct_ok = false;
  DBuf<float> m2m_part;             // FP32 M2M: each child's translated multipole (nboxes x NC)
  int p2p_tile = 0;                 // FP32 near-field staging shape (0 = default)
  int p2p_tile_user = 0, m2l_tile_user = 0;  // the caller's tile options (0 = tuned or default)
  DBuf<double> M64, L64;            // nboxes x NC
  DBuf<float> M32, L32;
  DBuf<float> Mhi, Mlo;             // split of M32 for the tensor-core M2L (TF32 or FP16 halves)
  DBuf<float> Mscale;               // FP16 form: power-of-two scale of each box's split multipole
  DBuf<int> dev_err;                // set by a bounded device wait that gave up
  DBuf<double> K64;                 // M2P coefficient sets of the W sources
  DBuf<float> K32;
  DBuf<double> far_acc, near_acc;   // FP64 path: 4 x n each, phi, gx, gy, gz (sorted order)
  DBuf<float4> far32;               // mixed path: the far field per sorted target
  DBuf<double> adj_grad_w, adj_grad_q;  // n x 3 (adjoint)
  DBuf<double> adj_phi;
  DBuf<double> host_io;             // device staging for fmm_solve_host

  // profiler: CUDA events around each pass on the plan's stream
  bool prof_on = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  struct ProfRec {
    int pass;
    cudaEvent_t a, b;
  };
  std::vector<ProfRec> prof_recs;
  int64_t prof_launches[kNumPasses] = {};
  cudaEvent_t next_event() {
    if (ev_used == ev_pool.size()) {
      cudaEvent_t e;
      FMM_CUDA(cudaEventCreate(&e));
      ev_pool.push_back(e);
    }
    return ev_pool[ev_used++];
  }

  // CUDA graph of one eval (+ adjoint) for fixed buffers; dropped on rebuild
  cudaGraphExec_t graph_exec = nullptr;
  const void *graph_key[8] = {};

  // scratch
  DBuf<int32_t> s_i32a, s_i32b, s_i32c, s_i32d, s_hist, s_scan;
  DBuf<uint64_t> s_u64a, s_u64b;
  DBuf<int32_t> s_total;            // device scalars for scan totals
  DBuf<int32_t> ca_off, ca_idx;     // coarser-or-equal adjacent leaves per box

  HelmholtzState helm;
};

// Records CUDA events around one pass when the plan's profiler is on.
struct PassScope {
  fmm_plan_impl &P;
  int pass;
  cudaEvent_t a = nullptr;
  uint64_t l0 = 0;
  PassScope(fmm_plan_impl &p, int ps) : P(p), pass(ps) {
    if (!P.prof_on) return;
    a = P.next_event();
    FMM_CUDA(cudaEventRecord(a, P.stream));
    l0 = launch_count();
  }
  ~PassScope() {
    if (!a) return;
    cudaEvent_t b = nullptr;
    try {
      b = P.next_event();
    } catch (...) {
      return;
    }
    if (cudaEventRecord(b, P.stream) != cudaSuccess) return;
    P.prof_recs.push_back({pass, a, b});
    P.prof_launches[pass] += (int64_t)(launch_count() - l0);
  }
};

// tree.cu
void build_tree(fmm_plan_impl &P, const double *d_xyz, int64_t n);
// root cube + Morton keys into caller memory: partial holds 7 x 1024 doubles,
// geom 8 doubles (lo[3], D, non-finite flag); perm gets the identity
void morton_keys_raw(const double *d_xyz, int64_t n, double *partial, double *geom, uint64_t *keys,
                     int32_t *perm, cudaStream_t s);
void set_points(fmm_plan_impl &P, const double *d_xyz);
// the V-list CSR of a plan whose M2L does not need it (on request; synchronous)
void build_vlists(fmm_plan_impl &P);
// M2L tiles of the boxes of level >= 2 and, in mixed precision, their source tables
void build_m2l_tiles(fmm_plan_impl &P);
// dual.cu: cell radii, the dual-tree walk, and its M2L / P2P lists
void build_dual_lists(fmm_plan_impl &P);
// operators.cu
void build_operators(fmm_plan_impl &P);
// rotated M2L tables (operators.cu); a no-op unless P.m2l_rot
void build_rotation(fmm_plan_impl &P);
size_t rotation_entries(int p);  // sum_n (2n+1)^2 over n <= p
// m2l.cu
void build_m2l_tables(fmm_plan_impl &P);
// m2l_tc.cu
size_t m2l_tc_operator_floats(int p);
size_t m2l_tc_pitch(int p);  // row pitch (values) of the split multipoles
void pack_m2l_tc_operators(int p, const double *m2l_in_major, float *out);
size_t m2l_tc16_operator_halves(int p);
void pack_m2l_tc16_operators(int p, const double *m2l_in_major, uint16_t *out, float *rowscale,
                             float *colscale);
// tune.cu: fastest leaf size for these points (cached per size bucket, order, precision)
int tuned_leaf_size(fmm_plan_impl &P, const double *d_xyz, int64_t n);
// eval.cu
void eval_fmm(fmm_plan_impl &P, const double *d_q, double *d_phi, double *d_grad);
void adjoint_fmm(fmm_plan_impl &P, const double *d_w, const double *d_q, const double *d_grad_q,
                 double *d_dq, double *d_dx);
void release_plan(fmm_plan_impl &P);
// helmholtz.cu: phi = sum_j q_j e^{i kappa |x_i - x_j|} / |x_i - x_j| (complex,
// interleaved, input order), and the release of its buffers
void eval_helmholtz(fmm_plan_impl &P, double kappa, int p, const double *d_q, double *d_phi);
void release_helmholtz(fmm_plan_impl &P);
void drop_graph(fmm_plan_impl &P);

// read a device int32 scalar (synchronous)
int32_t read_scalar(const int32_t *d, cudaStream_t s);

}  // namespace fmm

struct fmm_plan_s : fmm::fmm_plan_impl {};
