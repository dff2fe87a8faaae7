// eval_kernels.cuh -- launchers of the evaluation passes.
#pragma once
#include "plan.cuh"

namespace fmm {

template <typename T>
struct V4;
template <>
struct V4<double> {
  using type = Dbl4;
};
template <>
struct V4<float> {
  using type = float4;
};

template <typename T>
void launch_permute_charges(int64_t n, const int32_t *perm, const double *q,
                            const typename V4<T>::type *pl, typename V4<T>::type *src, cudaStream_t s);
template <typename T>
void launch_p2m(int p, int64_t nleaves, const int32_t *leaves, const int32_t *first,
                const int32_t *count, const BoxGeo *geo, const typename V4<T>::type *src, const double *side,
                T *M, double *M64, int coarse, cudaStream_t s);
template <typename T>
void launch_p2l(int p, int64_t nx, const int32_t *xboxes, const int32_t *xoff, const int32_t *xidx,
                const int32_t *first, const int32_t *count, const BoxGeo *geo,
                const typename V4<T>::type *src, const double *side, T *L, cudaStream_t s);
template <typename Tin, typename Tout, typename Top, typename Tacc>
void launch_m2m(int p, int32_t b0, int32_t nbl, const int32_t *child, const int32_t *nchild,
                const BoxGeo *geo, const Tin *Mc, const Top *ops, Tout *Mp, float *Mp32,
                cudaStream_t s);
template <typename Tself, typename Tpar, typename Tout, typename Top, typename Tacc>
void launch_l2l(int p, int32_t b0, int32_t nbl, const int32_t *parent, const BoxGeo *geo,
                const Tself *Lself, const Tpar *Lpar, const Top *ops, Tout *Lout, float *Lout32,
                cudaStream_t s);
template <typename Tin>
void launch_to_f64(int64_t count, const Tin *in, double *out, cudaStream_t s);
// lfar: leaves above this level get no far field (2 for U/V/W/X lists, 1
// for the dual tree).  far: per sorted target (phi, gx, gy, gz) at the
// evaluation's precision (FP32 for the mixed path: its far field is FP32
// arithmetic, so a wider store would add no accuracy)
template <typename T>
void launch_l2p(int p, int64_t nleaves, const int32_t *leaves, const int32_t *first,
                const int32_t *count, const BoxGeo *geo, const typename V4<T>::type *src, const double *side,
                const T *L, int64_t n, typename V4<T>::type *far, int lfar, cudaStream_t s);
// M2P over W lists; K is scratch of 4 * coef_pitch(p+1) per X box (the W sources)
template <typename T>
void launch_m2p(int p, int64_t nw, const int32_t *wleaves, const int32_t *woff, const int32_t *widx,
                int64_t nx, const int32_t *xboxes, const int32_t *xslot, const int32_t *first,
                const int32_t *count, const BoxGeo *geo, const typename V4<T>::type *src, const double *side,
                const T *M, T *K, int64_t n, typename V4<T>::type *far, cudaStream_t s);
// FP32 M2M into the parents [b0, b0 + nbl) of level l from the children of
// level l + 1 (oct_off / oct_order: boxes grouped by level and octant; part:
// nboxes x coef_pitch(p) scratch for the translated children)
void launch_m2m_f32q(int p, int l, int32_t b0, int32_t nbl, int32_t nchildren,
                     const int32_t *oct_off, const int32_t *oct_order, const int32_t *child,
                     const int32_t *nchild, const float *opT, float *part, float *M, cudaStream_t s);
// the boxes of levels [l0, nlevels) grouped by octant within each level
void launch_octant_groups(int nlevels, const int32_t *level_off_host, int32_t b0, int32_t nb,
                          const BoxGeo *geo, int32_t *oct_off, int32_t *oct_pos, int32_t *oct_order,
                          cudaStream_t s);
// FP32 L2L into the nbl boxes [b0, b0 + nbl) of level l from their parents
void launch_l2l_f32q(int p, int l, int32_t b0, int32_t nbl, const int32_t *oct_off,
                     const int32_t *oct_order, const int32_t *parent, const BoxGeo *geo,
                     const float *opT, float *L, cudaStream_t s);
void launch_combine(int64_t n, const int32_t *iperm, const double *far, const double *near,
                    double *phi, double *grad, cudaStream_t s);
void launch_adjoint_dx(int64_t n, const double *w, const double *q, const double *gq,
                       const double *gw, double *dx, cudaStream_t s);

// m2l.cu
template <typename T>
void launch_m2l(int p, int64_t ntiles, const M2LTile *tiles, int tile, const int32_t *order,
                const int32_t *voff, const int32_t *vidx, const BoxGeo *geo, const T *M,
                const T *ops, T *L, cudaStream_t s);

// rotated M2L over the per-tile source tables (any order up to kRotMaxOrder)
template <typename T>
void launch_m2l_rot(int p, int64_t ntiles, const M2LTile *tiles, int tile_size, const int32_t *table,
                    const int16_t *slots, const int32_t *nslots, const int32_t *order, const T *M,
                    const T *rot, const T *zt, T *L, cudaStream_t s);

void launch_m2l_staged(int p, int64_t ntiles, const M2LTile *tiles, const int32_t *table,
                       const int16_t *slots, const int32_t *nslots, const int32_t *order,
                       const float *M, const float *opsp, float *L, cudaStream_t s);

// m2l_tc.cu: splits M into Mhi/Mlo (pitch m2l_tc_pitch(p) values), then
// contracts on the tensor cores; err is set if a bounded wait gave up.
// TF32 form: Mhi/Mlo FP32 (TF32 values), opt from pack_m2l_tc_operators.
// FP16 form: Mhi/Mlo FP16, opt from pack_m2l_tc16_operators with its row and
// column scales, mscale one float per box (written by the split).
constexpr bool kM2LTcDefaultF16 = true;  // the form m2l_tile 0 selects
struct M2LTcForm {
  bool f16;
  void *Mhi, *Mlo;
  const void *opt;
  const float *rowscale, *colscale;
  float *mscale;
};
void launch_m2l_tc(int p, int64_t ntiles, const M2LTile *tiles, const int32_t *table,
                   const int16_t *slots, const int32_t *nslots, const int32_t *order, int64_t nb,
                   const float *M, const M2LTcForm &form, float *L, int *err, cudaStream_t s);

// dual.cu: M2L over the dual-tree pairs (cells of any two sizes); writes
// (or, with accumulate, adds to) L of every box
template <typename T>
void launch_m2l_dual(int p, int64_t nb, const int32_t *off, const int32_t *idx, const BoxGeo *geo,
                     const T *M, T *L, bool accumulate, cudaStream_t s);

// p2p.cu.  The FP32 path packs every leaf's sources in pairs once per
// evaluation into `pairs` (p2p_pair_floats(n) floats).  Once per plan,
// launch_p2p_meta writes one staging record per U entry (meta, meta_z: nu
// entries each) and a sort key per leaf (cost_key, cost_leaf: nleaves each,
// the key falling as the leaf's work grows); `order` is the leaves sorted by
// that key.  `tile` (1..p2p_num_tiles()) picks the staging shape; `ticket` is
// one device int of scratch; err is set if a bounded wait for a staging copy
// gave up.  The FP64 path uses none of them.
// The FP32 near field also finishes each target: it adds the far field
// (far, FP32 per sorted target) to its compensated near-field sum in FP64 and
// writes phi / grad at the target's input index perm[i] (grad may be NULL).
struct P2PScratch {
  float4 *pairs;
  const int4 *meta;
  const float *meta_z;
  const int32_t *order;
  int *ticket;
  int tile;
  int *err;
  const float4 *far;
  const int32_t *perm;
  double *phi, *grad;
};
size_t p2p_pair_floats(int64_t n);
int p2p_num_tiles();
constexpr int kP2PDefaultTile = 1;
void launch_p2p_meta(int64_t nleaves, const int32_t *leaves, const int32_t *uoff, const int32_t *uidx,
                     const int32_t *first, const int32_t *count, const BoxGeo *geo, const double *side,
                     int4 *meta, float *meta_z, uint64_t *cost_key, int32_t *cost_leaf, cudaStream_t s);
template <typename T>
void launch_p2p(int64_t nleaves, const int32_t *leaves, const int32_t *uoff, const int32_t *uidx,
                const int32_t *first, const int32_t *count, const BoxGeo *geo,
                const typename V4<T>::type *src, const double *side, int64_t n, double *near,
                P2PScratch *scratch, cudaStream_t s);

}  // namespace fmm
