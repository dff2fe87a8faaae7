// api.cu -- the C-ABI of libfmm (declared in include/fmm.h): argument
// checks, error mapping, the device memory pool, and plan lifetime.
#include <cmath>
#include <cstring>
#include <atomic>
#include <mutex>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "eval_kernels.cuh"

namespace fmm {

namespace {

thread_local std::string g_last_error;
std::atomic<uint64_t> g_launches{0};

cudaMemPool_t pool_for_current_device() {
  static std::mutex mu;
  static std::unordered_map<int, cudaMemPool_t> pools;
  int dev = 0;
  FMM_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  auto it = pools.find(dev);
  if (it != pools.end()) return it->second;
  cudaMemPoolProps props;
  std::memset(&props, 0, sizeof props);
  props.allocType = cudaMemAllocationTypePinned;
  props.handleTypes = cudaMemHandleTypeNone;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t pool;
  FMM_CUDA(cudaMemPoolCreate(&pool, &props));
  uint64_t keep = UINT64_MAX;  // keep freed memory for the next plan
  FMM_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
  pools[dev] = pool;
  return pool;
}

fmm_status fail(fmm_status s, const std::string &msg) {
  g_last_error = msg;
  return s;
}

template <typename F>
fmm_status guarded(F &&f) {
  try {
    f();
    return FMM_OK;
  } catch (const Error &e) {
    return fail(e.status, e.what());
  } catch (const std::bad_alloc &) {
    return fail(FMM_ERR_OOM, "host allocation failed");
  } catch (const std::exception &e) {
    return fail(FMM_ERR_CUDA, e.what());
  }
}

void check_opts(const fmm_opts *o) {
  if (!o) return;
  if (o->precision != FMM_FP64 && o->precision != FMM_MIXED)
    throw Error(FMM_ERR_INVALID_ARG, "opts.precision must be FMM_FP64 or FMM_MIXED");
  if (o->max_depth < 0 || o->max_depth > kMaxDepth)
    throw Error(FMM_ERR_INVALID_ARG, "opts.max_depth must be in 0..21");
  if (o->m2l_path < 0 || o->m2l_path > 3)
    throw Error(FMM_ERR_INVALID_ARG, "opts.m2l_path must be 0, 1, 2 or 3");
  if (o->interaction < 0 || o->interaction > 1)
    throw Error(FMM_ERR_INVALID_ARG, "opts.interaction must be 0 or 1");
  if (!(o->mac_theta >= 0.0 && o->mac_theta < 1.0))
    throw Error(FMM_ERR_INVALID_ARG, "opts.mac_theta must be in [0, 1)");
  if (o->m2l_tile < 0 || o->m2l_tile > 2)
    throw Error(FMM_ERR_INVALID_ARG, "opts.m2l_tile must be 0, 1 or 2");
  if (o->wx_direct < 0 || o->wx_direct > 1)
    throw Error(FMM_ERR_INVALID_ARG, "opts.wx_direct must be 0 or 1");
  if (o->p2p_tile < 0 || o->p2p_tile > p2p_num_tiles())
    throw Error(FMM_ERR_INVALID_ARG, "opts.p2p_tile must be in 0.." + std::to_string(p2p_num_tiles()));
}

void apply_opts(fmm_plan_impl &P, const fmm_opts *o) {
  if (!o) return;
  P.m2l_path = o->m2l_path;
  P.precision = o->precision;
  P.coarse_fp64_levels = o->coarse_fp64_levels == 0 ? 3 : o->coarse_fp64_levels;
  P.max_depth = o->max_depth == 0 ? kMaxDepth : o->max_depth;
  P.dual = o->interaction == 1;
  P.theta = o->mac_theta > 0.0 ? o->mac_theta : 0.5;
  P.p2p_tile = P.p2p_tile_user = o->p2p_tile;
  P.m2l_tile = P.m2l_tile_user = o->m2l_tile;
  P.wx_direct_max = o->wx_direct && !P.dual ? (P.order + 1) * (P.order + 1) : 0;
}

}  // namespace

fmm_status record_error(fmm_status s, const std::string &msg) { return fail(s, msg); }

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
uint64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }

void *device_alloc(size_t bytes, cudaStream_t s) {
  if (bytes == 0) bytes = 16;
  void *p = nullptr;
  cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, pool_for_current_device(), s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Error(e == cudaErrorMemoryAllocation ? FMM_ERR_OOM : FMM_ERR_CUDA,
                std::string("device allocation of ") + std::to_string(bytes) +
                    " bytes failed: " + cudaGetErrorString(e));
  }
  return p;
}

void device_free(void *p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

void drop_graph(fmm_plan_impl &P) {
  if (P.graph_exec) cudaGraphExecDestroy(P.graph_exec);
  P.graph_exec = nullptr;
  for (auto &k : P.graph_key) k = nullptr;
}

void release_plan(fmm_plan_impl &P) {
  drop_graph(P);
  for (auto &e : P.copy_ev)
    if (e) {
      cudaEventDestroy(e);
      e = nullptr;
    }
  if (P.copy_stream) {
    cudaStreamDestroy(P.copy_stream);
    P.copy_stream = nullptr;
  }
  P.geom.release(); P.partial.release(); P.keys.release(); P.keys_tmp.release();
  P.perm.release(); P.perm_tmp.release(); P.xyz_sorted.release(); P.pl64.release();
  P.pl32.release(); P.box_key.release(); P.box_level.release(); P.box_first.release();
  P.box_count.release(); P.box_parent.release(); P.box_child.release(); P.box_nchild.release();
  P.box_geo.release(); P.colleagues.release(); P.ncolleagues.release(); P.u_off.release();
  P.u_idx.release(); P.v_off.release(); P.v_idx.release(); P.w_off.release(); P.w_idx.release();
  P.x_off.release(); P.x_idx.release(); P.leaves.release(); P.xboxes.release();
  P.wleaves.release(); P.m2l_order.release(); P.m2l_tiles.release(); P.ops.m2l64.release();
  P.ops.m2m64.release(); P.ops.l2l64.release(); P.ops.m2l32.release(); P.ops.m2m32.release();
  P.ops.l2l32.release(); P.src64.release(); P.src32.release(); P.M64.release(); P.L64.release();
  P.M32.release(); P.L32.release(); P.far_acc.release(); P.near_acc.release();
  P.adj_grad_w.release(); P.adj_grad_q.release(); P.adj_phi.release(); P.host_io.release();
  P.s_i32a.release(); P.s_i32b.release(); P.s_i32c.release(); P.s_i32d.release();
  P.s_hist.release();
  P.s_scan.release(); P.s_u64a.release(); P.s_u64b.release(); P.s_total.release();
  P.ca_off.release(); P.ca_idx.release(); P.m2l_src.release(); P.m2l_slots.release();
  P.m2l_nslots.release(); P.ops.m2l32p.release(); P.ops.m2l_tc.release(); P.Mhi.release();
  P.Mlo.release(); P.dev_err.release(); P.Mscale.release(); P.ops.m2l_tc16.release();
  P.ops.m2l_tc16_rows.release(); P.ops.m2l_tc16_cols.release();
  P.xslot.release(); P.K64.release(); P.K32.release(); P.box_prob.release();
  P.box_side.release(); P.prob_off.release(); P.prob_geom.release(); P.iperm.release();
  P.ops.m2m32t.release(); P.ops.l2l32t.release();
  P.radius.release(); P.dt_a.release(); P.dt_b.release(); P.dt_m2l.release();
  P.dt_p2p.release(); P.dt_cnt.release(); P.dt_toff.release(); P.dt_tidx.release();
  P.dt_goff.release(); P.dt_gidx.release(); P.p2p_pairs.release(); P.p2p_meta.release(); P.p2p_meta_z.release();
  P.p2p_key.release(); P.p2p_key_tmp.release(); P.p2p_order.release(); P.p2p_order_tmp.release();
  P.p2p_ticket.release();
  P.oct_off.release(); P.oct_order.release(); P.oct_pos.release(); P.m2m_part.release();
  P.far32.release();
  release_helmholtz(P);
}

}  // namespace fmm

using namespace fmm;

extern "C" {

fmm_status fmm_plan_create(const double *d_xyz, int64_t n, int leaf_size, int order,
                           const fmm_opts *opts, void *stream, fmm_plan_t *out) {
  if (!out) return fail(FMM_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n < 0 || n >= (int64_t(1) << 31)) return fail(FMM_ERR_INVALID_ARG, "n must be in [0, 2^31)");
  if (leaf_size < 0) return fail(FMM_ERR_INVALID_ARG, "leaf_size must be >= 1 (or 0: autotune)");
  if (order < 0 || order > kMaxOrder) return fail(FMM_ERR_INVALID_ARG, "order must be in 0..20");
  if (n > 0 && !d_xyz) return fail(FMM_ERR_INVALID_ARG, "d_xyz is NULL");
  fmm_plan_s *P = nullptr;
  fmm_status st = guarded([&] {
    check_opts(opts);
    P = new fmm_plan_s();
    P->order = order;
    P->leaf_size = leaf_size > 0 ? leaf_size : 64;
    P->autotune = leaf_size == 0;
    P->stream = (cudaStream_t)stream;
    apply_opts(*P, opts);
    if (P->autotune && n > 0) P->leaf_size = tuned_leaf_size(*P, d_xyz, n);
    build_tree(*P, d_xyz, n);
  });
  if (st != FMM_OK) {
    if (P) {
      release_plan(*P);
      cudaStreamSynchronize(P->stream);
      delete P;
    }
    return st;
  }
  *out = P;
  return FMM_OK;
}

fmm_status fmm_plan_create_batch(const double *d_xyz, const int64_t *h_offsets, int nproblems,
                                 int leaf_size, int order, const fmm_opts *opts, void *stream,
                                 fmm_plan_t *out) {
  if (!out) return fail(FMM_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (nproblems < 1 || !h_offsets) return fail(FMM_ERR_INVALID_ARG, "need nproblems >= 1 and offsets");
  if (h_offsets[0] != 0) return fail(FMM_ERR_INVALID_ARG, "offsets[0] must be 0");
  for (int b = 0; b < nproblems; ++b)
    if (h_offsets[b + 1] < h_offsets[b]) return fail(FMM_ERR_INVALID_ARG, "offsets must not decrease");
  const int64_t n = h_offsets[nproblems];
  if (n >= (int64_t(1) << 31)) return fail(FMM_ERR_INVALID_ARG, "total points must be < 2^31");
  if (leaf_size < 0) return fail(FMM_ERR_INVALID_ARG, "leaf_size must be >= 1 (or 0: autotune)");
  if (order < 0 || order > kMaxOrder) return fail(FMM_ERR_INVALID_ARG, "order must be in 0..20");
  if (n > 0 && !d_xyz) return fail(FMM_ERR_INVALID_ARG, "d_xyz is NULL");
  fmm_plan_s *P = nullptr;
  fmm_status st = guarded([&] {
    check_opts(opts);
    P = new fmm_plan_s();
    P->order = order;
    P->leaf_size = leaf_size > 0 ? leaf_size : 64;
    P->autotune = leaf_size == 0;
    P->stream = (cudaStream_t)stream;
    P->nproblems = nproblems;
    P->prob_off_h.assign(h_offsets, h_offsets + nproblems + 1);
    apply_opts(*P, opts);
    if (P->autotune && n > 0) P->leaf_size = tuned_leaf_size(*P, d_xyz, n);
    build_tree(*P, d_xyz, n);
  });
  if (st != FMM_OK) {
    if (P) {
      release_plan(*P);
      cudaStreamSynchronize(P->stream);
      delete P;
    }
    return st;
  }
  *out = P;
  return FMM_OK;
}

fmm_status fmm_plan_rebuild(fmm_plan_t plan, const double *d_xyz, int64_t n, void *stream) {
  if (!plan) return fail(FMM_ERR_INVALID_ARG, "plan is NULL");
  if (n < 0 || n >= (int64_t(1) << 31)) return fail(FMM_ERR_INVALID_ARG, "n must be in [0, 2^31)");
  if (n > 0 && !d_xyz) return fail(FMM_ERR_INVALID_ARG, "d_xyz is NULL");
  if (plan->nproblems > 1 && n != plan->prob_off_h.back())
    return fail(FMM_ERR_INVALID_ARG, "a batch plan rebuilds only for the same problem sizes");
  return guarded([&] {
    plan->stream = (cudaStream_t)stream;
    if (plan->autotune && n > 0) plan->leaf_size = tuned_leaf_size(*plan, d_xyz, n);
    build_tree(*plan, d_xyz, n);
  });
}

fmm_status fmm_plan_set_points(fmm_plan_t plan, const double *d_xyz, void *stream) {
  if (!plan) return fail(FMM_ERR_INVALID_ARG, "plan is NULL");
  if (plan->n > 0 && !d_xyz) return fail(FMM_ERR_INVALID_ARG, "d_xyz is NULL");
  return guarded([&] {
    plan->stream = (cudaStream_t)stream;
    set_points(*plan, d_xyz);
  });
}

fmm_status fmm_eval(fmm_plan_t plan, const double *d_q, double *d_phi, double *d_grad,
                    void *stream) {
  if (!plan) return fail(FMM_ERR_INVALID_ARG, "plan is NULL");
  if (plan->n > 0 && (!d_q || !d_phi)) return fail(FMM_ERR_INVALID_ARG, "d_q or d_phi is NULL");
  return guarded([&] {
    plan->stream = (cudaStream_t)stream;
    eval_fmm(*plan, d_q, d_phi, d_grad);
  });
}

fmm_status fmm_helmholtz_eval(fmm_plan_t plan, double kappa, int order, const double *d_q,
                              double *d_phi, void *stream) {
  if (!plan) return fail(FMM_ERR_INVALID_ARG, "plan is NULL");
  if (plan->n > 0 && (!d_q || !d_phi)) return fail(FMM_ERR_INVALID_ARG, "d_q or d_phi is NULL");
  return guarded([&] {
    plan->stream = (cudaStream_t)stream;
    eval_helmholtz(*plan, kappa, order, d_q, d_phi);
  });
}

fmm_status fmm_adjoint(fmm_plan_t plan, const double *d_w, const double *d_q,
                       const double *d_grad_q, double *d_dq, double *d_dx, void *stream) {
  if (!plan) return fail(FMM_ERR_INVALID_ARG, "plan is NULL");
  if (plan->n > 0 && (!d_w || !d_dq || (d_dx && !d_q)))
    return fail(FMM_ERR_INVALID_ARG, "d_w, d_dq, or d_q (needed for d_dx) is NULL");
  return guarded([&] {
    plan->stream = (cudaStream_t)stream;
    adjoint_fmm(*plan, d_w, d_q, d_grad_q, d_dq, d_dx);
  });
}

fmm_status fmm_eval_graph(fmm_plan_t plan, const double *d_q, double *d_phi, double *d_grad,
                          const double *d_w, double *d_dq, double *d_dx, void *stream) {
  if (!plan) return fail(FMM_ERR_INVALID_ARG, "plan is NULL");
  if (!stream) return fail(FMM_ERR_INVALID_ARG, "fmm_eval_graph needs a non-default stream");
  if (plan->n > 0 && (!d_q || !d_phi)) return fail(FMM_ERR_INVALID_ARG, "d_q or d_phi is NULL");
  if (plan->n > 0 && d_w && !d_dq) return fail(FMM_ERR_INVALID_ARG, "d_dq is NULL");
  return guarded([&] {
    cudaStream_t s = (cudaStream_t)stream;
    plan->stream = s;
    if (plan->n == 0) return;
    const void *key[8] = {d_q, d_phi, d_grad, d_w, d_dq, d_dx, nullptr, nullptr};
    bool same = plan->graph_exec != nullptr;
    for (int i = 0; i < 8 && same; ++i) same = key[i] == plan->graph_key[i];
    if (!same) {
      drop_graph(*plan);
      // one eager pass sizes every buffer and builds the operators, so the
      // captured work allocates nothing and never synchronises
      auto work = [&] {
        eval_fmm(*plan, d_q, d_phi, d_grad);
        if (d_w) adjoint_fmm(*plan, d_w, d_q, d_grad, d_dq, d_dx);
      };
      work();
      const bool prof = plan->prof_on;
      plan->prof_on = false;
      cudaGraph_t g = nullptr;
      FMM_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      try {
        work();
      } catch (...) {
        cudaStreamEndCapture(s, &g);
        if (g) cudaGraphDestroy(g);
        plan->prof_on = prof;
        throw;
      }
      plan->prof_on = prof;
      FMM_CUDA(cudaStreamEndCapture(s, &g));
      cudaError_t e = cudaGraphInstantiate(&plan->graph_exec, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        plan->graph_exec = nullptr;
        throw Error(FMM_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
      }
      for (int i = 0; i < 8; ++i) plan->graph_key[i] = key[i];
    }
    FMM_CUDA(cudaGraphLaunch(plan->graph_exec, s));
  });
}

fmm_status fmm_solve_host(fmm_plan_t plan, const double *h_xyz, const double *h_q, int64_t n,
                          double *h_phi, double *h_grad, void *stream) {
  if (!plan) return fail(FMM_ERR_INVALID_ARG, "plan is NULL");
  if (n < 0 || n >= (int64_t(1) << 31)) return fail(FMM_ERR_INVALID_ARG, "n must be in [0, 2^31)");
  if (n > 0 && (!h_xyz || !h_q || !h_phi)) return fail(FMM_ERR_INVALID_ARG, "a host pointer is NULL");
  if (plan->nproblems > 1 && n != plan->prob_off_h.back())
    return fail(FMM_ERR_INVALID_ARG, "a batch plan solves only for the same problem sizes");
  return guarded([&] {
    cudaStream_t s = (cudaStream_t)stream;
    plan->stream = s;
    if (n == 0) {
      build_tree(*plan, nullptr, 0);
      return;
    }
    fmm_plan_impl &P = *plan;
    if (!P.copy_stream) FMM_CUDA(cudaStreamCreateWithFlags(&P.copy_stream, cudaStreamNonBlocking));
    for (auto &e : P.copy_ev)
      if (!e) FMM_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    cudaStream_t c = P.copy_stream;
    P.host_io.resize(8 * (size_t)n, s);
    double *d_xyz = P.host_io.p, *d_q = d_xyz + 3 * n, *d_phi = d_q + n, *d_grad = d_phi + n;
    // the coordinates first, alone; the charges on the side stream while the
    // tree is built (after the staging buffer exists and the coordinates landed)
    FMM_CUDA(cudaMemcpyAsync(d_xyz, h_xyz, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s));
    FMM_CUDA(cudaEventRecord(P.copy_ev[0], s));
    FMM_CUDA(cudaStreamWaitEvent(c, P.copy_ev[0], 0));
    FMM_CUDA(cudaMemcpyAsync(d_q, h_q, sizeof(double) * n, cudaMemcpyHostToDevice, c));
    FMM_CUDA(cudaEventRecord(P.copy_ev[3], c));
    build_tree(P, d_xyz, n);
    FMM_CUDA(cudaStreamWaitEvent(s, P.copy_ev[3], 0));  // q has landed
    eval_fmm(P, d_q, d_phi, h_grad ? d_grad : nullptr);
    FMM_CUDA(cudaMemcpyAsync(h_phi, d_phi, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    if (h_grad)
      FMM_CUDA(cudaMemcpyAsync(h_grad, d_grad, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s));
    FMM_CUDA(cudaStreamSynchronize(s));
  });
}

fmm_status fmm_solve_adjoint_host(fmm_plan_t plan, const double *h_xyz, const double *h_q,
                                  const double *h_w, int64_t n, double *h_phi, double *h_grad,
                                  double *h_dq, double *h_dx, void *stream) {
  if (!plan) return fail(FMM_ERR_INVALID_ARG, "plan is NULL");
  if (n < 0 || n >= (int64_t(1) << 31)) return fail(FMM_ERR_INVALID_ARG, "n must be in [0, 2^31)");
  if (n > 0 && (!h_xyz || !h_q || !h_w || !h_phi || !h_grad || !h_dq || !h_dx))
    return fail(FMM_ERR_INVALID_ARG, "a host pointer is NULL");
  if (plan->nproblems > 1 && n != plan->prob_off_h.back())
    return fail(FMM_ERR_INVALID_ARG, "a batch plan solves only for the same problem sizes");
  return guarded([&] {
    cudaStream_t s = (cudaStream_t)stream;
    plan->stream = s;
    if (n == 0) {
      build_tree(*plan, nullptr, 0);
      return;
    }
    fmm_plan_impl &P = *plan;
    if (!P.copy_stream) FMM_CUDA(cudaStreamCreateWithFlags(&P.copy_stream, cudaStreamNonBlocking));
    for (auto &e : P.copy_ev)
      if (!e) FMM_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    cudaStream_t c = P.copy_stream;
    // device staging: xyz 3n, q n, w n | phi n, grad 3n, dq n, dx 3n
    P.host_io.resize(13 * (size_t)n, s);
    double *d_xyz = P.host_io.p, *d_q = d_xyz + 3 * n, *d_w = d_q + n;
    double *d_phi = d_w + n, *d_grad = d_phi + n, *d_dq = d_grad + 3 * n, *d_dx = d_dq + n;
    // the coordinates go up first, alone (the tree needs them); the charges
    // and the loss weights follow on the side stream while the tree is built
    // (the side stream starts after the staging buffer exists and the
    // coordinates have landed: stream order on s)
    FMM_CUDA(cudaMemcpyAsync(d_xyz, h_xyz, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s));
    FMM_CUDA(cudaEventRecord(P.copy_ev[0], s));
    FMM_CUDA(cudaStreamWaitEvent(c, P.copy_ev[0], 0));
    FMM_CUDA(cudaMemcpyAsync(d_q, h_q, sizeof(double) * n, cudaMemcpyHostToDevice, c));
    FMM_CUDA(cudaEventRecord(P.copy_ev[3], c));
    FMM_CUDA(cudaMemcpyAsync(d_w, h_w, sizeof(double) * n, cudaMemcpyHostToDevice, c));
    FMM_CUDA(cudaEventRecord(P.copy_ev[1], c));
    build_tree(P, d_xyz, n);
    FMM_CUDA(cudaStreamWaitEvent(s, P.copy_ev[3], 0));  // q has landed
    eval_fmm(P, d_q, d_phi, d_grad);
    // phi and grad come down while the adjoint runs (it only reads d_grad)
    FMM_CUDA(cudaEventRecord(P.copy_ev[2], s));
    FMM_CUDA(cudaStreamWaitEvent(c, P.copy_ev[2], 0));
    FMM_CUDA(cudaMemcpyAsync(h_phi, d_phi, sizeof(double) * n, cudaMemcpyDeviceToHost, c));
    FMM_CUDA(cudaMemcpyAsync(h_grad, d_grad, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, c));
    FMM_CUDA(cudaStreamWaitEvent(s, P.copy_ev[1], 0));  // w has landed
    adjoint_fmm(P, d_w, d_q, d_grad, d_dq, d_dx);
    FMM_CUDA(cudaMemcpyAsync(h_dq, d_dq, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    FMM_CUDA(cudaMemcpyAsync(h_dx, d_dx, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s));
    FMM_CUDA(cudaStreamSynchronize(c));
    FMM_CUDA(cudaStreamSynchronize(s));
  });
}

fmm_status fmm_plan_tiles(fmm_plan_t plan, int *p2p_tile, int *m2l_tile) {
  if (!plan) return fail(FMM_ERR_INVALID_ARG, "plan is NULL");
  if (p2p_tile) *p2p_tile = plan->p2p_tile > 0 ? plan->p2p_tile : kP2PDefaultTile;
  if (m2l_tile) *m2l_tile = plan->m2l_tile > 0 ? plan->m2l_tile : (kM2LTcDefaultF16 ? 2 : 1);
  return FMM_OK;
}

fmm_status fmm_plan_sizes(fmm_plan_t plan, int64_t sizes[10]) {
  if (!plan || !sizes) return fail(FMM_ERR_INVALID_ARG, "plan or sizes is NULL");
  if (!plan->v_built) {
    fmm_status st = guarded([&] { build_vlists(*plan); });
    if (st != FMM_OK) return st;
  }
  sizes[0] = plan->n;
  sizes[1] = plan->nboxes;
  sizes[2] = plan->nlevels;
  sizes[3] = plan->nu;
  sizes[4] = plan->nv;
  sizes[5] = plan->nw;
  sizes[6] = plan->nx;
  sizes[7] = plan->order;
  sizes[8] = plan->leaf_size;
  sizes[9] = plan->precision;
  return FMM_OK;
}

fmm_status fmm_plan_export(fmm_plan_t plan, int which, void *h_dst, size_t bytes) {
  if (!plan) return fail(FMM_ERR_INVALID_ARG, "plan is NULL");
  if (!plan->v_built && (which == 12 || which == 13)) {
    fmm_status st = guarded([&] { build_vlists(*plan); });
    if (st != FMM_OK) return st;
  }
  const fmm_plan_impl &P = *plan;
  const void *src = nullptr;
  size_t want = 0;
  const size_t n = (size_t)P.n, nb = (size_t)P.nboxes, nb1 = nb + 1;
  bool lists = nb > 0;
  std::vector<double> geo4;
  for (int b = 0; b < P.nproblems; ++b)
    for (int a = 0; a < 4; ++a)
      geo4.push_back(P.prob_geom_h.size() >= (size_t)8 * (b + 1) ? P.prob_geom_h[8 * b + a]
                                                                  : (a == 3 ? 1.0 : 0.0));
  switch (which) {
    case 0: src = P.keys.p; want = n * 8; break;
    case 1: src = P.perm.p; want = n * 4; break;
    case 2: src = nullptr; want = P.level_off.size() * 4; break;
    case 3: src = P.box_key.p; want = nb * 8; break;
    case 4: src = P.box_level.p; want = nb * 4; break;
    case 5: src = P.box_first.p; want = nb * 4; break;
    case 6: src = P.box_count.p; want = nb * 4; break;
    case 7: src = P.box_parent.p; want = nb * 4; break;
    case 8: src = P.box_child.p; want = nb * 4; break;
    case 9: src = P.box_nchild.p; want = nb * 4; break;
    case 10: src = P.u_off.p; want = lists ? nb1 * 4 : 0; break;
    case 11: src = P.u_idx.p; want = (size_t)P.nu * 4; break;
    case 12: src = P.v_off.p; want = lists ? nb1 * 4 : 0; break;
    case 13: src = P.v_idx.p; want = (size_t)P.nv * 4; break;
    case 14: src = P.w_off.p; want = lists ? nb1 * 4 : 0; break;
    case 15: src = P.w_idx.p; want = (size_t)P.nw * 4; break;
    case 16: src = P.x_off.p; want = lists ? nb1 * 4 : 0; break;
    case 17: src = P.x_idx.p; want = (size_t)P.nx * 4; break;
    case 18: src = nullptr; want = geo4.size() * sizeof(double); break;
    case 19: src = nullptr; want = (P.prob_off_h.empty() ? 2 : P.prob_off_h.size()) * sizeof(int64_t); break;
    case 20: src = P.radius.p; want = P.dual ? nb * 8 : 0; break;
    default: return fail(FMM_ERR_INVALID_ARG, "unknown export array");
  }
  if (bytes != want)
    return fail(FMM_ERR_INVALID_ARG, "export: bytes must be " + std::to_string(want));
  if (want == 0) return FMM_OK;
  if (!h_dst) return fail(FMM_ERR_INVALID_ARG, "h_dst is NULL");
  if (which == 2) {
    std::memcpy(h_dst, P.level_off.data(), want);
    return FMM_OK;
  }
  if (which == 18) {
    std::memcpy(h_dst, geo4.data(), want);
    return FMM_OK;
  }
  if (which == 19) {
    std::vector<int64_t> off = P.prob_off_h.empty() ? std::vector<int64_t>{0, P.n} : P.prob_off_h;
    std::memcpy(h_dst, off.data(), want);
    return FMM_OK;
  }
  return guarded([&] {
    FMM_CUDA(cudaStreamSynchronize(P.stream));
    FMM_CUDA(cudaMemcpy(h_dst, src, want, cudaMemcpyDeviceToHost));
  });
}

fmm_status fmm_profile(fmm_plan_t plan, int enable) {
  if (!plan) return fail(FMM_ERR_INVALID_ARG, "plan is NULL");
  plan->prof_on = enable != 0;
  return FMM_OK;
}

fmm_status fmm_profile_read(fmm_plan_t plan, double ms[FMM_NPASS], int64_t launches[FMM_NPASS]) {
  if (!plan || !ms || !launches) return fail(FMM_ERR_INVALID_ARG, "plan, ms or launches is NULL");
  return guarded([&] {
    FMM_CUDA(cudaStreamSynchronize(plan->stream));
    for (int i = 0; i < FMM_NPASS; ++i) {
      ms[i] = 0.0;
      launches[i] = plan->prof_launches[i];
      plan->prof_launches[i] = 0;
    }
    for (const auto &r : plan->prof_recs) {
      float t = 0.f;
      FMM_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
      ms[r.pass] += t;
    }
    plan->prof_recs.clear();
    plan->ev_used = 0;
  });
}

uint64_t fmm_kernel_launches(void) { return launch_count(); }

fmm_status fmm_memory_usage(uint64_t *current, uint64_t *peak, int reset_peak) {
  return guarded([&] {
    cudaMemPool_t pool = pool_for_current_device();
    uint64_t c = 0, h = 0;
    FMM_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &c));
    FMM_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &h));
    if (current) *current = c;
    if (peak) *peak = h;
    if (reset_peak) {
      uint64_t z = 0;
      FMM_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &z));
    }
  });
}

fmm_status fmm_sync(fmm_plan_t plan, void *stream) {
  if (!plan) return fail(FMM_ERR_INVALID_ARG, "plan is NULL");
  fmm_status st = FMM_OK;
  fmm_status g = guarded([&] {
    cudaStream_t s = (cudaStream_t)stream;
    FMM_CUDA(cudaStreamSynchronize(s));
    if (plan->dev_err.p) {
      int h = 0;
      FMM_CUDA(cudaMemcpy(&h, plan->dev_err.p, sizeof(int), cudaMemcpyDeviceToHost));
      if (h) {
        FMM_CUDA(cudaMemset(plan->dev_err.p, 0, sizeof(int)));
        st = fail(FMM_ERR_TIMEOUT, "a bounded device-side wait gave up (tensor-core M2L)");
      }
    }
  });
  return g != FMM_OK ? g : st;
}

fmm_status fmm_plan_destroy(fmm_plan_t plan) {
  if (!plan) return FMM_OK;
  fmm_status st = guarded([&] {
    release_plan(*plan);
    FMM_CUDA(cudaStreamSynchronize(plan->stream));
    for (cudaEvent_t e : plan->ev_pool) cudaEventDestroy(e);
  });
  delete plan;
  return st;
}

const char *fmm_status_string(fmm_status s) {
  switch (s) {
    case FMM_OK: return "FMM_OK";
    case FMM_ERR_INVALID_ARG: return "FMM_ERR_INVALID_ARG";
    case FMM_ERR_CUDA: return "FMM_ERR_CUDA";
    case FMM_ERR_OOM: return "FMM_ERR_OOM";
    case FMM_ERR_TIMEOUT: return "FMM_ERR_TIMEOUT";
    case FMM_ERR_NONFINITE_INPUT: return "FMM_ERR_NONFINITE_INPUT";
    case FMM_ERR_UNSUPPORTED: return "FMM_ERR_UNSUPPORTED";
  }
  return "FMM_ERR_UNKNOWN";
}

const char *fmm_last_error_message(void) { return g_last_error.c_str(); }

}  // extern "C"
