// eval.cu -- the FMM mat-vec pass sequence on one stream (§1: matrix-free
// H^2 mat-vec; §2.2 translation operators and near field):
//   permute charges -> P2M -> M2M (deepest parents first) -> M2L over all
//   levels >= 2 -> P2L -> L2L (top-down) -> L2P -> M2P -> P2P -> FP64
//   per-target reduction and scatter to the caller's order.
// FP64 mode runs every pass in FP64.  Mixed mode runs P2M/M2L/P2L/L2P/M2P/P2P
// in FP32 and keeps FP64 only for M2M/L2L into the coarsest levels
// (<= coarse_fp64_levels) and for the per-target totals.
// A dual-tree plan runs the same sequence with M2M up to level 1, one M2L
// launch over its accepted pairs (any level, writes every box's local), L2L
// from level 1 down, no P2L/M2P, and P2P over its leaf pairs.
#include "eval_kernels.cuh"
#include <algorithm>

#include "m2l_config.cuh"
#include "sort.cuh"

namespace fmm {

namespace {

void ensure_workspace(fmm_plan_impl &P, bool need64, bool need32) {
  const size_t nc = (size_t)coef_pitch(P.order);  // row pitch of the coefficient arrays
  const size_t nb = (size_t)P.nboxes;
  cudaStream_t s = P.stream;
  if (need32) {  // mixed: the far field in FP32; the near field finishes each target
    P.far32.resize((size_t)P.n, s);
  } else {
    P.far_acc.resize(4 * (size_t)P.n, s);
    P.near_acc.resize(4 * (size_t)P.n, s);
  }
  if (need64) {
    P.M64.resize(nb * nc, s);
    P.L64.resize(nb * nc, s);
  }
  if (need32) {
    P.M32.resize(nb * nc, s);
    P.L32.resize(nb * nc, s);
  }
}

void eval_fp64(fmm_plan_impl &P, const double *d_q, double *d_phi, double *d_grad) {
  const int p = P.order;
  const int64_t n = P.n;
  cudaStream_t s = P.stream;
  ensure_workspace(P, true, false);
  P.src64.resize(n, s);
  {
    PassScope ps_(P, kPassP2M);
    launch_permute_charges<double>(n, P.perm.p, d_q, P.pl64.p, P.src64.p, s);
    launch_p2m<double>(p, P.nleaves, P.leaves.p, P.box_first.p, P.box_count.p, P.box_geo.p,
                       P.src64.p, P.box_side.p, P.M64.p, nullptr, -1, s);
  }
  const int ltop = P.dual ? 1 : 2;  // coarsest level whose boxes take part in M2L
  for (int l = P.nlevels - 2; l >= ltop; --l) {
    PassScope ps_(P, kPassM2M);
    launch_m2m<double, double, double, double>(p, P.level_off[l], P.level_off[l + 1] - P.level_off[l],
                                               P.box_child.p, P.box_nchild.p, P.box_geo.p, P.M64.p,
                                               P.ops.m2m64.p, P.M64.p, nullptr, s);
  }
  {
    PassScope ps_(P, kPassM2L);
    if (P.dual)
      launch_m2l_dual<double>(p, P.nboxes, P.v_off.p, P.v_idx.p, P.box_geo.p, P.M64.p, P.L64.p,
                              false, s);
    else if (P.m2l_rot)
      launch_m2l_rot<double>(p, P.nm2l_tiles, P.m2l_tiles.p, P.m2l_tile_size, P.m2l_src.p,
                             P.m2l_slots.p, P.m2l_nslots.p, P.m2l_order.p, P.M64.p, P.ops.rot64.p,
                             P.ops.zt64.p, P.L64.p, s);
    else
      launch_m2l<double>(p, P.nm2l_tiles, P.m2l_tiles.p, P.m2l_tile_size, P.m2l_order.p, P.v_off.p,
                         P.v_idx.p, P.box_geo.p, P.M64.p, P.ops.m2l64.p, P.L64.p, s);
  }
  {
    PassScope ps_(P, kPassP2L);
    launch_p2l<double>(p, P.nxboxes, P.xboxes.p, P.x_off.p, P.x_idx.p, P.box_first.p, P.box_count.p,
                       P.box_geo.p, P.src64.p, P.box_side.p, P.L64.p, s);
  }
  for (int l = ltop + 1; l < P.nlevels; ++l) {
    PassScope ps_(P, kPassL2L);
    launch_l2l<double, double, double, double, double>(
        p, P.level_off[l], P.level_off[l + 1] - P.level_off[l], P.box_parent.p, P.box_geo.p, P.L64.p,
        P.L64.p, P.ops.l2l64.p, P.L64.p, nullptr, s);
  }
  {
    PassScope ps_(P, kPassL2P);
    launch_l2p<double>(p, P.nleaves, P.leaves.p, P.box_first.p, P.box_count.p, P.box_geo.p, P.src64.p,
                       P.box_side.p, P.L64.p, n, reinterpret_cast<Dbl4 *>(P.far_acc.p), ltop, s);
  }
  if (P.nwleaves > 0) {
    PassScope ps_(P, kPassM2P);
    P.K64.resize(std::max<size_t>(1, (size_t)P.nxboxes * 4 * coef_pitch(p + 1)), s);
    launch_m2p<double>(p, P.nwleaves, P.wleaves.p, P.w_off.p, P.w_idx.p, P.nxboxes, P.xboxes.p,
                       P.xslot.p, P.box_first.p, P.box_count.p, P.box_geo.p, P.src64.p, P.box_side.p, P.M64.p,
                       P.K64.p, n, reinterpret_cast<Dbl4 *>(P.far_acc.p), s);
  }
  {
    PassScope ps_(P, kPassP2P);
    launch_p2p<double>(P.nleaves, P.leaves.p, P.u_off.p, P.u_idx.p, P.box_first.p, P.box_count.p,
                       P.box_geo.p, P.src64.p, P.box_side.p, n, P.near_acc.p, nullptr, s);
  }
  {
    PassScope ps_(P, kPassReduce);
    launch_combine(n, P.iperm.p, P.far_acc.p, P.near_acc.p, d_phi, d_grad, s);
  }
}

// The tensor-core M2L's operand form (TF32 or FP16 split) and its buffers.
M2LTcForm tc_form(fmm_plan_impl &P) {
  cudaStream_t s = P.stream;
  const size_t nb = (size_t)P.nboxes, kt = m2l_tc_pitch(P.order);
  const bool f16 = P.m2l_tile == 0 ? kM2LTcDefaultF16 : P.m2l_tile == 2;
  const size_t words = f16 ? kt / 2 : kt;  // floats per box and half
  P.Mhi.resize(nb * words, s);
  P.Mlo.resize(nb * words, s);
  if (f16) P.Mscale.resize(nb, s);
  return {f16, P.Mhi.p, P.Mlo.p,
          f16 ? static_cast<const void *>(P.ops.m2l_tc16.p) : static_cast<const void *>(P.ops.m2l_tc.p),
          P.ops.m2l_tc16_rows.p, P.ops.m2l_tc16_cols.p, P.Mscale.p};
}

// Once per plan, for the FP32 near field: the staging record of every U entry
// and the leaves sorted by decreasing work class (targets x sources).  Plan work:
// the profiler books it under the lists.
void prepare_p2p_f32(fmm_plan_impl &P) {
  if (P.p2p_meta_ok) return;
  cudaStream_t s = P.stream;
  PassScope ps_(P, kPassLists);
  const size_t nl = std::max<int64_t>(P.nleaves, 1);
  P.p2p_meta.resize(std::max<int64_t>(P.nu, 1), s);
  P.p2p_meta_z.resize(std::max<int64_t>(P.nu, 1), s);
  P.p2p_key.resize(nl, s);
  P.p2p_order.resize(nl, s);
  P.p2p_ticket.resize(1, s);
  launch_p2p_meta(P.nleaves, P.leaves.p, P.u_off.p, P.u_idx.p, P.box_first.p, P.box_count.p,
                  P.box_geo.p, P.box_side.p, P.p2p_meta.p, P.p2p_meta_z.p, P.p2p_key.p,
                  P.p2p_order.p, s);
  radix_sort(P.p2p_key, P.p2p_order, P.p2p_key_tmp, P.p2p_order_tmp, P.nleaves, digit_shifts(0, 16),
             P.s_hist, P.s_scan, s);
  P.p2p_meta_ok = true;
}

// Once per plan, for the FP32 M2M / L2L: the boxes of each level grouped by
// their octant within the parent (plan work: the profiler books it under the
// lists), and the scratch of the children's translated multipoles.
void prepare_oct_groups(fmm_plan_impl &P) {
  if (P.oct_ok) return;
  cudaStream_t s = P.stream;
  PassScope ps_(P, kPassLists);
  const size_t nb = std::max<int64_t>(P.nboxes, 1);
  P.oct_off.resize((size_t)9 * std::max(P.nlevels, 1), s);
  P.oct_order.resize(nb, s);
  P.oct_pos.resize(nb, s);
  P.m2m_part.resize(nb * (size_t)coef_pitch(P.order), s);
  launch_octant_groups(P.nlevels, P.level_off.data(), 0, (int32_t)P.nboxes, P.box_geo.p,
                       P.oct_off.p, P.oct_pos.p, P.oct_order.p, s);
  P.oct_ok = true;
}

void eval_mixed(fmm_plan_impl &P, const double *d_q, double *d_phi, double *d_grad) {
  const int p = P.order;
  const int64_t n = P.n;
  cudaStream_t s = P.stream;
  const int lc = P.coarse_fp64_levels;  // M2M/L2L into levels <= lc in FP64
  const bool coarse = lc >= 2;
  ensure_workspace(P, coarse, true);
  prepare_p2p_f32(P);
  prepare_oct_groups(P);
  P.src32.resize(n, s);
  {
    PassScope ps_(P, kPassP2M);
    launch_permute_charges<float>(n, P.perm.p, d_q, P.pl32.p, P.src32.p, s);
    launch_p2m<float>(p, P.nleaves, P.leaves.p, P.box_first.p, P.box_count.p, P.box_geo.p, P.src32.p,
                      P.box_side.p, P.M32.p, coarse ? P.M64.p : nullptr, lc, s);
  }
  const int ltop = P.dual ? 1 : 2;  // coarsest level whose boxes take part in M2L
  for (int l = P.nlevels - 2; l >= ltop; --l) {
    const int32_t b0 = P.level_off[l], nbl = P.level_off[l + 1] - b0;
    PassScope ps_(P, kPassM2M);
    if (l <= lc) {
      if (l + 1 <= lc)
        launch_m2m<double, double, double, double>(p, b0, nbl, P.box_child.p, P.box_nchild.p,
                                                   P.box_geo.p, P.M64.p, P.ops.m2m64.p, P.M64.p,
                                                   P.M32.p, s);
      else
        launch_m2m<float, double, double, double>(p, b0, nbl, P.box_child.p, P.box_nchild.p,
                                                  P.box_geo.p, P.M32.p, P.ops.m2m64.p, P.M64.p,
                                                  P.M32.p, s);
    } else {
      launch_m2m_f32q(p, l, b0, nbl, P.level_off[l + 2] - P.level_off[l + 1], P.oct_off.p,
                      P.oct_order.p, P.box_child.p, P.box_nchild.p, P.ops.m2m32t.p,
                      P.m2m_part.p, P.M32.p, s);
    }
  }
  {
    PassScope ps_(P, kPassM2L);
    if (P.dual && p > kM2LStagedMaxOrder) {
      launch_m2l_dual<float>(p, P.nboxes, P.v_off.p, P.v_idx.p, P.box_geo.p, P.M32.p, P.L32.p,
                             false, s);
    } else if (P.dual) {
      // the pairs of the fixed-offset tiles on the tensor cores (they write L
      // of every box of level >= 2), levels 0 and 1 cleared, then the rest
      const size_t ldc = (size_t)coef_pitch(p);
      const size_t b2 = (size_t)(P.nlevels > 2 ? P.level_off[2] : P.nboxes);
      FMM_CUDA(cudaMemsetAsync(P.L32.p, 0, sizeof(float) * b2 * ldc, s));
      if (P.m2l_tc) {
        launch_m2l_tc(p, P.nm2l_tiles, P.m2l_tiles.p, P.m2l_src.p, P.m2l_slots.p, P.m2l_nslots.p,
                      P.m2l_order.p, P.nboxes, P.M32.p, tc_form(P), P.L32.p, P.dev_err.p, s);
      } else {
        launch_m2l_staged(p, P.nm2l_tiles, P.m2l_tiles.p, P.m2l_src.p, P.m2l_slots.p,
                          P.m2l_nslots.p, P.m2l_order.p, P.M32.p, P.ops.m2l32p.p, P.L32.p, s);
      }
      launch_m2l_dual<float>(p, P.nboxes, P.dt_goff.p, P.dt_gidx.p, P.box_geo.p, P.M32.p, P.L32.p,
                             true, s);
    } else if (P.m2l_rot) {
      launch_m2l_rot<float>(p, P.nm2l_tiles, P.m2l_tiles.p, P.m2l_tile_size, P.m2l_src.p,
                            P.m2l_slots.p, P.m2l_nslots.p, P.m2l_order.p, P.M32.p, P.ops.rot32.p,
                            P.ops.zt32.p, P.L32.p, s);
    } else if (P.m2l_tc) {
      launch_m2l_tc(p, P.nm2l_tiles, P.m2l_tiles.p, P.m2l_src.p, P.m2l_slots.p, P.m2l_nslots.p,
                    P.m2l_order.p, P.nboxes, P.M32.p, tc_form(P), P.L32.p, P.dev_err.p, s);
    } else if (p <= kM2LStagedMaxOrder)
      launch_m2l_staged(p, P.nm2l_tiles, P.m2l_tiles.p, P.m2l_src.p, P.m2l_slots.p, P.m2l_nslots.p,
                        P.m2l_order.p, P.M32.p, P.ops.m2l32p.p, P.L32.p, s);
    else
      launch_m2l<float>(p, P.nm2l_tiles, P.m2l_tiles.p, P.m2l_tile_size, P.m2l_order.p, P.v_off.p,
                        P.v_idx.p, P.box_geo.p, P.M32.p, P.ops.m2l32.p, P.L32.p, s);
  }
  {
    PassScope ps_(P, kPassP2L);
    launch_p2l<float>(p, P.nxboxes, P.xboxes.p, P.x_off.p, P.x_idx.p, P.box_first.p, P.box_count.p,
                      P.box_geo.p, P.src32.p, P.box_side.p, P.L32.p, s);
  }
  const size_t nc = (size_t)coef_pitch(p);
  if (coarse && P.nlevels > ltop) {
    const size_t b0 = (size_t)P.level_off[ltop], b1 = (size_t)P.level_off[ltop + 1];
    PassScope ps_(P, kPassL2L);
    launch_to_f64<float>((int64_t)((b1 - b0) * nc), P.L32.p + b0 * nc, P.L64.p + b0 * nc, s);
  }
  for (int l = ltop + 1; l < P.nlevels; ++l) {
    const int32_t b0 = P.level_off[l], nbl = P.level_off[l + 1] - b0;
    PassScope ps_(P, kPassL2L);
    if (l <= lc)
      launch_l2l<float, double, double, double, double>(p, b0, nbl, P.box_parent.p, P.box_geo.p,
                                                        P.L32.p, P.L64.p, P.ops.l2l64.p, P.L64.p,
                                                        P.L32.p, s);
    else
      launch_l2l_f32q(p, l, b0, nbl, P.oct_off.p, P.oct_order.p, P.box_parent.p, P.box_geo.p,
                      P.ops.l2l32t.p, P.L32.p, s);
  }
  {
    PassScope ps_(P, kPassL2P);
    launch_l2p<float>(p, P.nleaves, P.leaves.p, P.box_first.p, P.box_count.p, P.box_geo.p, P.src32.p,
                      P.box_side.p, P.L32.p, n, P.far32.p, ltop, s);
  }
  if (P.nwleaves > 0) {
    PassScope ps_(P, kPassM2P);
    P.K32.resize(std::max<size_t>(1, (size_t)P.nxboxes * 4 * coef_pitch(p + 1)), s);
    launch_m2p<float>(p, P.nwleaves, P.wleaves.p, P.w_off.p, P.w_idx.p, P.nxboxes, P.xboxes.p,
                      P.xslot.p, P.box_first.p, P.box_count.p, P.box_geo.p, P.src32.p, P.box_side.p, P.M32.p,
                      P.K32.p, n, P.far32.p, s);
  }
  {
    PassScope ps_(P, kPassP2P);
    P.p2p_pairs.resize(p2p_pair_floats(n), s);
    P2PScratch scratch{reinterpret_cast<float4 *>(P.p2p_pairs.p), P.p2p_meta.p, P.p2p_meta_z.p,
                       P.p2p_order.p, P.p2p_ticket.p, P.p2p_tile > 0 ? P.p2p_tile : kP2PDefaultTile,
                       P.dev_err.p, P.far32.p, P.perm.p, d_phi, d_grad};
    launch_p2p<float>(P.nleaves, P.leaves.p, P.u_off.p, P.u_idx.p, P.box_first.p, P.box_count.p,
                      P.box_geo.p, P.src32.p, P.box_side.p, n, nullptr, &scratch, s);
  }
}

}  // namespace

void eval_fmm(fmm_plan_impl &P, const double *d_q, double *d_phi, double *d_grad) {
  if (P.n == 0) return;
  build_operators(P);
  build_rotation(P);
  if (!P.dev_err.p) {
    P.dev_err.resize(1, P.stream);
    FMM_CUDA(cudaMemsetAsync(P.dev_err.p, 0, sizeof(int), P.stream));
  }
  if (P.precision == FMM_FP64) eval_fp64(P, d_q, d_phi, d_grad);
  else eval_mixed(P, d_q, d_phi, d_grad);
}

void adjoint_fmm(fmm_plan_impl &P, const double *d_w, const double *d_q, const double *d_grad_q,
                 double *d_dq, double *d_dx) {
  const int64_t n = P.n;
  if (n == 0) return;
  cudaStream_t s = P.stream;
  P.adj_grad_w.resize(3 * (size_t)n, s);
  // dL/dq = A~^T w = A~ w (the truncated operator is symmetric)
  eval_fmm(P, d_w, d_dq, d_dx ? P.adj_grad_w.p : nullptr);
  if (!d_dx) return;
  const double *gq = d_grad_q;
  if (!gq) {  // recompute instead of store
    P.adj_grad_q.resize(3 * (size_t)n, s);
    P.adj_phi.resize((size_t)n, s);
    eval_fmm(P, d_q, P.adj_phi.p, P.adj_grad_q.p);
    gq = P.adj_grad_q.p;
  }
  {
    PassScope ps_(P, kPassReduce);
    launch_adjoint_dx(n, d_w, d_q, gq, P.adj_grad_w.p, d_dx, s);
  }
}

}  // namespace fmm
