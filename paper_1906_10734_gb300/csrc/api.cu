// C ABI entry points of libhpm (declared in include/hpm.h).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "hpm_internal.cuh"

namespace hpm {

static thread_local char g_cuda_err[256] = "no error";

const char *set_cuda_error(cudaError_t e) {
  snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
  return g_cuda_err;
}

static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[kMaxDevices] = {};

hpm_status lib_pool(cudaMemPool_t *out) {
  int dev = 0;
  HPM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return HPM_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_pool_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    HPM_CUDA(cudaMemPoolCreate(&pool, &props));
    // keep freed blocks in this pool between solves instead of returning them
    // to the driver at every synchronisation
    uint64_t thr = UINT64_MAX;
    HPM_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
    g_pool[dev] = pool;
  }
  *out = g_pool[dev];
  return HPM_OK;
}

hpm_status lib_malloc_async(void **p, size_t bytes, cudaStream_t s) {
  cudaMemPool_t pool = nullptr;
  HPM_TRY(lib_pool(&pool));
  const cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, s);
  if (e != cudaSuccess) {
    set_cuda_error(e);
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? HPM_ERR_OOM : HPM_ERR_CUDA;
  }
  return HPM_OK;
}

hpm_status DevBuf::ensure(size_t bytes, cudaStream_t s, bool keep) {
  used = std::max(used, bytes);
  if (bytes <= cap && p) return HPM_OK;
  size_t ncap = bytes + bytes / 4 + 256;
  void *np = nullptr;
  HPM_TRY(lib_malloc_async(&np, ncap, s));
  if (keep && p && cap) HPM_CUDA(cudaMemcpyAsync(np, p, cap, cudaMemcpyDeviceToDevice, s));
  if (p) HPM_CUDA(cudaFreeAsync(p, s));
  p = np;
  cap = ncap;
  return HPM_OK;
}

void DevBuf::release(cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
  p = nullptr;
  cap = 0;
  used = 0;
}

// Gridlet constants (Sec. 2.2 nodes, Sec. 2.3 child-to-parent), FP64 -> FP32,
// for the Ng nodes x_j = (j + 1/2)/Ng - 1/2 widened by `ext` nodes of the same
// spacing on each side (Sec. 2.5; ext = 0: the gridlet itself): tb.ng = Ng + 2 ext.
static void make_tables(int ng0, int ext, GridletTables &tb) {
  memset(&tb, 0, sizeof(tb));
  const int ng = ng0 + 2 * ext;
  tb.ng = ng;
  double x[kMaxNg];
  for (int j = 0; j < ng; ++j) x[j] = (j - ext + 0.5) / ng0 - 0.5;
  for (int j = 0; j < ng; ++j) {
    double den = 1.0;
    for (int k = 0; k < ng; ++k)
      if (k != j) den *= x[j] - x[k];
    tb.node[j] = (float)x[j];
    tb.node_d[j] = x[j];
    tb.inv_den_d[j] = 1.0 / den;
    tb.inv_den[j] = (float)(1.0 / den);
    tb.node_lo[j] = (float)(x[j] - (double)tb.node[j]);
    tb.inv_den_lo[j] = (float)(1.0 / den - (double)tb.inv_den[j]);
    double den_u = 1.0;
    for (int k = 0; k < ng; ++k)
      if (k != j) den_u *= (double)(2 * (j - k));
    tb.inv_den_u[j] = 1.0 / den_u;
  }
  for (int s = 0; s < 2; ++s) {
    const double a = s ? 0.5 : -0.5;
    for (int p = 0; p < ng; ++p)
      for (int q = 0; q < ng; ++q) {
        const double t = (a + x[q]) / 2.0;
        double v = 1.0;
        for (int k = 0; k < ng; ++k)
          if (k != p) v *= (t - x[k]) / (x[p] - x[k]);
        tb.t1[s][p][q] = (float)v;
        tb.t1lo[s][p][q] = (float)(v - (double)tb.t1[s][p][q]);
      }
  }
}

// The plan's device buffers: first the plan-time tables (the Green
// transforms and lattice, W and its exponents, the near-field table), then
// the buffers of the tree build and the solve (the host_io ones stage
// hpm_solve_host's and the batch's inputs and outputs on the device).
constexpr int kPlanTables = 9;
template <class F>
static void for_each_buf(hpm_plan_s *pl, F &&f) {
  DevBuf *bufs[] = {&pl->ghat, &pl->kx_green, &pl->kz_green, &pl->tc_w, &pl->tc_wexp, &pl->glat, &pl->near_tab,
                    &pl->tc_mean, &pl->gmean,
                    &pl->t.keys, &pl->t.keys_alt, &pl->t.perm, &pl->t.perm_alt, &pl->t.spm, &pl->t.pbox,
                    &pl->t.box_key, &pl->t.box_beg, &pl->t.box_end, &pl->t.box_parent, &pl->t.box_flags,
                    &pl->t.box_child, &pl->t.box_nb, &pl->t.cnt, &pl->t.off, &pl->t.bnd, &pl->t.par_box, &pl->t.tgt_blk, &pl->t.tgt_info, &pl->t.tc_rows, &pl->t.tc_tgt, &pl->t.tgt_box,
                    &pl->t.box_tgt, &pl->t.leaf_box, &pl->t.p2g_box, &pl->t.item_leaf, &pl->t.item_s0,
                    &pl->t.item_s1, &pl->t.item_t, &pl->t.leaf_nitem, &pl->t.leaf_ns, &pl->t.big_leaf, &pl->t.split_leaf, &pl->t.leaf_item0, &pl->t.leaf_part0, &pl->s.part, &pl->t.err, &pl->t.lvl_dev, &pl->t.counters, &pl->t.scan_buf,
                    &pl->s.grid, &pl->s.m2l_raw, &pl->s.loc, &pl->s.locc, &pl->s.m2lc, &pl->s.far, &pl->s.m2l_scratch, &pl->s.work, &pl->s.grid_hl, &pl->s.box_em, &pl->s.col_exp, &pl->s.zone_mass, &pl->s.level_amax,
                    &pl->batch_desc, &pl->t.offsets,
                    &pl->host_io_pos, &pl->host_io_mass, &pl->host_io_phi, &pl->host_io_acc};
  constexpr int nb = (int)(sizeof(bufs) / sizeof(bufs[0]));
  for (int i = 0; i < nb; ++i) f(bufs[i], i < kPlanTables ? 0 : 1);
}

static void release_all(hpm_plan_s *pl, cudaStream_t s) {
  for_each_buf(pl, [s](DevBuf *b, int) { b->release(s); });
}

// A tree build starts a new count of what the work buffers need.
void reset_work_need(hpm_plan_s *pl) {
  for_each_buf(pl, [](DevBuf *b, int kind) {
    if (kind) b->used = 0;
  });
}

// Device bytes of the plan: its tables (held), and what the last build and
// solve needed of the per-input buffers.
void plan_bytes(hpm_plan_s *pl, int64_t *tables, int64_t *work) {
  int64_t t = 0, w = 0;
  for_each_buf(pl, [&](DevBuf *b, int kind) {
    if (kind == 0) t += (int64_t)b->cap;
    else w += (int64_t)b->used;
  });
  *tables = t;
  *work = w;
}

}  // namespace hpm

using namespace hpm;

extern "C" {

const char *hpm_status_str(hpm_status s) {
  switch (s) {
    case HPM_OK: return "ok";
    case HPM_ERR_INVALID_ARG: return "invalid argument";
    case HPM_ERR_OUT_OF_DOMAIN: return "particle outside the domain";
    case HPM_ERR_OOM: return "out of device memory";
    case HPM_ERR_CUDA: return "CUDA error";
    case HPM_ERR_TIMEOUT: return "bounded wait timed out";
    case HPM_ERR_NOT_BUILT: return "tree not built";
    case HPM_ERR_BUSY: return "busy";
    case HPM_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char *hpm_last_cuda_error(void) { return g_cuda_err; }

hpm_status hpm_plan(const hpm_domain *dom, int max_depth, int gridlet_order, const hpm_green *green,
                    const hpm_plan_opts *opts, hpm_plan_t *out) {
  if (!dom || !green || !out) return HPM_ERR_INVALID_ARG;
  *out = nullptr;
  if (max_depth < 0 || max_depth > kMaxDepth) return HPM_ERR_INVALID_ARG;
  if (gridlet_order < 1 || gridlet_order > kMaxNg) return HPM_ERR_INVALID_ARG;
  if (!(dom->side > 0.0) || !std::isfinite(dom->side)) return HPM_ERR_INVALID_ARG;
  for (int d = 0; d < 3; ++d)
    if (!std::isfinite(dom->origin[d])) return HPM_ERR_INVALID_ARG;
  switch (green->kind) {
    case HPM_GREEN_PLUMMER:
    case HPM_GREEN_YUKAWA:
      if (!(green->eps >= 0.0) || !std::isfinite(green->eps)) return HPM_ERR_INVALID_ARG;
      if (green->kind == HPM_GREEN_YUKAWA && (!(green->lambda > 0.0) || !std::isfinite(green->lambda)))
        return HPM_ERR_INVALID_ARG;
      break;
    case HPM_GREEN_NEWTON:
      break;
    case HPM_GREEN_USER:
      if (!green->user_g) return HPM_ERR_INVALID_ARG;
      break;
    default:
      return HPM_ERR_UNSUPPORTED;
  }
  if (opts && opts->leaf_max < 0) return HPM_ERR_INVALID_ARG;
  if (opts && (opts->flags & HPM_FLAG_EXTENDED_GRIDLET) && gridlet_order + 2 > kMaxNg) return HPM_ERR_UNSUPPORTED;
  hpm_plan_s *pl = new (std::nothrow) hpm_plan_s();
  if (!pl) return HPM_ERR_OOM;
  pl->dom = *dom;
  pl->max_depth = max_depth;
  pl->ng = gridlet_order;
  pl->green = *green;
  if (pl->green.kind == HPM_GREEN_NEWTON) pl->green.eps = 0.0;
  pl->opts = opts ? *opts : hpm_plan_opts{0, 0};
  cudaGetDevice(&pl->device);
  make_tables(gridlet_order, 0, pl->tab);
  const int ext = (pl->opts.flags & HPM_FLAG_EXTENDED_GRIDLET) ? 1 : 0;
  make_tables(gridlet_order, ext, pl->tab_loc);
  pl->ng_loc = gridlet_order + 2 * ext;
  hpm_status s = precompute_green(pl, 0);
  if (s == HPM_OK) s = tc_precompute(pl, 0);
  if (s == HPM_OK) {
    cudaError_t e = cudaStreamSynchronize(0);
    if (e != cudaSuccess) {
      set_cuda_error(e);
      s = HPM_ERR_CUDA;
    }
  }
  if (s == HPM_OK && (pl->opts.flags & 1)) {
    for (auto &ev : pl->ev)
      if (cudaEventCreate(&ev) != cudaSuccess) s = HPM_ERR_CUDA;
    pl->events_ready = s == HPM_OK;
  }
  if (s != HPM_OK) {
    release_all(pl, 0);
    delete pl;
    return s;
  }
  *out = pl;
  return HPM_OK;
}

hpm_status hpm_build_tree(hpm_plan_t plan, const double *d_pos, int64_t n, void *stream) {
  if (!plan || n < 0 || n >= (int64_t)1 << 31 || (n > 0 && !d_pos)) return HPM_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (plan->events_ready) cudaEventRecord(plan->ev[8], st);
  hpm_status s = build_tree(plan, d_pos, n, nullptr, 1, st);
  if (plan->events_ready) cudaEventRecord(plan->ev[9], st);
  return s;
}

hpm_status hpm_build_tree_batch(hpm_plan_t plan, const double *d_pos, const int64_t *h_offsets, int n_problems,
                                void *stream) {
  if (!plan || !h_offsets || n_problems < 1) return HPM_ERR_INVALID_ARG;
  if (h_offsets[0] != 0) return HPM_ERR_INVALID_ARG;
  for (int p = 0; p < n_problems; ++p)
    if (h_offsets[p + 1] < h_offsets[p]) return HPM_ERR_INVALID_ARG;
  const int64_t n = h_offsets[n_problems];
  if (n >= (int64_t)1 << 31 || (n > 0 && !d_pos)) return HPM_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (plan->events_ready) cudaEventRecord(plan->ev[8], st);
  hpm_status s = build_tree(plan, d_pos, n, h_offsets, n_problems, st);
  if (plan->events_ready) cudaEventRecord(plan->ev[9], st);
  if (s == HPM_OK) plan->prob_off.assign(h_offsets, h_offsets + n_problems + 1);
  return s;
}

hpm_status hpm_solve_batch(hpm_plan_t plan, const hpm_problem *h_problems, int n_problems, void *stream) {
  if (!plan || !h_problems || n_problems < 1) return HPM_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<int64_t> off(n_problems + 1, 0);
  for (int p = 0; p < n_problems; ++p) {
    if (h_problems[p].n < 0 || (h_problems[p].n > 0 && (!h_problems[p].d_pos || !h_problems[p].d_mass)))
      return HPM_ERR_INVALID_ARG;
    off[p + 1] = off[p] + h_problems[p].n;
  }
  const int64_t n = off[n_problems];
  if (n >= (int64_t)1 << 31) return HPM_ERR_INVALID_ARG;
  const size_t nn = n > 0 ? (size_t)n : 1;
  HPM_TRY(plan->host_io_pos.ensure(sizeof(double) * 3 * nn, st));
  HPM_TRY(plan->host_io_mass.ensure(sizeof(double) * nn, st));
  HPM_TRY(plan->host_io_phi.ensure(sizeof(float) * nn, st));
  HPM_TRY(plan->host_io_acc.ensure(sizeof(float) * 3 * nn, st));
  HPM_TRY(plan->batch_desc.ensure(sizeof(hpm_problem) * n_problems + sizeof(int64_t) * (n_problems + 1), st));
  hpm_problem *d_desc = plan->batch_desc.as<hpm_problem>();
  int64_t *d_off = reinterpret_cast<int64_t *>(d_desc + n_problems);
  HPM_CUDA(cudaMemcpyAsync(d_desc, h_problems, sizeof(hpm_problem) * n_problems, cudaMemcpyHostToDevice, st));
  HPM_CUDA(cudaMemcpyAsync(d_off, off.data(), sizeof(int64_t) * (n_problems + 1), cudaMemcpyHostToDevice, st));
  HPM_TRY(batch_gather(d_desc, d_off, n_problems, n, plan->host_io_pos.as<double>(), plan->host_io_mass.as<double>(),
                       st));
  HPM_TRY(hpm_build_tree_batch(plan, plan->host_io_pos.as<double>(), off.data(), n_problems, stream));
  HPM_TRY(hpm_solve(plan, plan->host_io_pos.as<double>(), plan->host_io_mass.as<double>(),
                    plan->host_io_phi.as<float>(), plan->host_io_acc.as<float>(), stream));
  HPM_TRY(batch_scatter(d_desc, d_off, n_problems, n, plan->host_io_phi.as<float>(), plan->host_io_acc.as<float>(),
                        st));
  return HPM_OK;
}

hpm_status hpm_solve(hpm_plan_t plan, const double *d_pos, const double *d_mass, float *d_phi, float *d_acc,
                     void *stream) {
  if (!plan) return HPM_ERR_INVALID_ARG;
  if (!plan->built) return HPM_ERR_NOT_BUILT;
  if (plan->n > 0 && (!d_pos || !d_mass)) return HPM_ERR_INVALID_ARG;
  return solve(plan, d_pos, d_mass, d_phi, d_acc, (cudaStream_t)stream);
}

// The solves' error word (a bounded device wait that ran out): read after the
// stream has drained, cleared once reported.
// The solve's error word: its copy to the host is enqueued on `st` (through
// the plan's pinned read-back buffer where the build allocated it), read after
// the caller's synchronisation; a timeout is reported once and cleared.
static int *enqueue_solve_error(hpm_plan_t plan, cudaStream_t st, int *local, hpm_status *s) {
  *local = 0;
  *s = HPM_OK;
  if (!plan->t.err.p) return local;
  int *he = plan->h_pin ? reinterpret_cast<int *>(plan->h_pin + 768) : local;
  const cudaError_t e = cudaMemcpyAsync(he, plan->t.err.as<int>() + 1, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) {
    hpm::set_cuda_error(e);
    *s = HPM_ERR_CUDA;
  }
  return he;
}
static hpm_status solve_error_status(hpm_plan_t plan, int e, cudaStream_t st) {
  if (!(e & hpm::kErrTimeout)) return HPM_OK;
  HPM_CUDA(cudaMemsetAsync(plan->t.err.as<int>() + 1, 0, sizeof(int), st));
  HPM_CUDA(cudaStreamSynchronize(st));
  return HPM_ERR_TIMEOUT;
}
static hpm_status take_solve_error(hpm_plan_t plan, cudaStream_t st) {
  int local = 0;
  hpm_status s = HPM_OK;
  const int *he = enqueue_solve_error(plan, st, &local, &s);
  HPM_TRY(s);
  HPM_CUDA(cudaStreamSynchronize(st));
  return solve_error_status(plan, *he, st);
}

hpm_status hpm_solve_host(hpm_plan_t plan, const double *h_pos, const double *h_mass, int64_t n, float *h_phi,
                          float *h_acc, void *stream) {
  if (!plan || n < 0 || (n > 0 && (!h_pos || !h_mass))) return HPM_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t nn = n > 0 ? (size_t)n : 1;
  HPM_TRY(plan->host_io_pos.ensure(sizeof(double) * 3 * nn, st));
  HPM_TRY(plan->host_io_mass.ensure(sizeof(double) * nn, st));
  HPM_TRY(plan->host_io_phi.ensure(sizeof(float) * nn, st));
  HPM_TRY(plan->host_io_acc.ensure(sizeof(float) * 3 * nn, st));
  if (n > 0) {
    if (!plan->io_stream) {
      HPM_CUDA(cudaStreamCreateWithFlags(&plan->io_stream, cudaStreamNonBlocking));
      for (auto &ev : plan->io_ev) HPM_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    }
    HPM_CUDA(cudaMemcpyAsync(plan->host_io_pos.p, h_pos, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st));
    // the masses follow the positions on the copy engine but are first needed
    // by the solve, so their copy overlaps the tree build
    HPM_CUDA(cudaEventRecord(plan->io_ev[0], st));
    HPM_CUDA(cudaStreamWaitEvent(plan->io_stream, plan->io_ev[0], 0));
    HPM_CUDA(cudaMemcpyAsync(plan->host_io_mass.p, h_mass, sizeof(double) * n, cudaMemcpyHostToDevice,
                             plan->io_stream));
    HPM_CUDA(cudaEventRecord(plan->io_ev[1], plan->io_stream));
  }
  hpm_status s = hpm_build_tree(plan, plan->host_io_pos.as<double>(), n, stream);
  if (n > 0) {
    const cudaError_t e = cudaStreamWaitEvent(st, plan->io_ev[1], 0);
    if (e != cudaSuccess && s == HPM_OK) {
      hpm::set_cuda_error(e);
      s = HPM_ERR_CUDA;
    }
  }
  if (s == HPM_OK)
    s = hpm_solve(plan, plan->host_io_pos.as<double>(), plan->host_io_mass.as<double>(),
                  plan->host_io_phi.as<float>(), plan->host_io_acc.as<float>(), stream);
  if (s != HPM_OK) {
    // no copy from the caller's buffers may outlive the call
    if (n > 0) cudaStreamSynchronize(plan->io_stream);
    return s;
  }
  if (n > 0 && h_phi)
    HPM_CUDA(cudaMemcpyAsync(h_phi, plan->host_io_phi.p, sizeof(float) * n, cudaMemcpyDeviceToHost, st));
  if (n > 0 && h_acc)
    HPM_CUDA(cudaMemcpyAsync(h_acc, plan->host_io_acc.p, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost, st));
  // the error word rides on the same synchronisation as the results
  int local = 0;
  hpm_status es = HPM_OK;
  const int *he = enqueue_solve_error(plan, st, &local, &es);
  HPM_CUDA(cudaStreamSynchronize(st));
  HPM_TRY(es);
  return solve_error_status(plan, *he, st);
}

hpm_status hpm_get_lists_info(hpm_plan_t plan, hpm_lists_info *info) {
  if (!plan || !info) return HPM_ERR_INVALID_ARG;
  if (!plan->built) return HPM_ERR_NOT_BUILT;
  info->n_particles = plan->n;
  info->n_cells = plan->ncell;
  info->n_targets = plan->ntgt;
  info->n_leaves = plan->nleaf;
  info->n_boxes = plan->nbox;
  info->max_depth = plan->max_depth;
  info->depth_reached = plan->n > 0 ? plan->depth_reached : -1;
  return HPM_OK;
}

hpm_status hpm_get_lists(hpm_plan_t plan, int32_t *level, uint64_t *key, int64_t *begin, int64_t *end,
                         uint8_t *leaf, uint64_t *iz, uint32_t *near, int64_t *perm) {
  if (!plan) return HPM_ERR_INVALID_ARG;
  if (!plan->built) return HPM_ERR_NOT_BUILT;
  HPM_CUDA(cudaDeviceSynchronize());
  const int64_t nb = plan->nbox, n = plan->n;
  if (n == 0) return HPM_OK;
  std::vector<uint64_t> bk(nb);
  std::vector<int> bb(nb), be(nb), bp(nb), bc(nb * 8), bn(nb * 27);
  std::vector<uint8_t> bf(nb);
  TreeDev &t = plan->t;
  HPM_CUDA(cudaMemcpy(bk.data(), t.box_key.p, sizeof(uint64_t) * nb, cudaMemcpyDeviceToHost));
  HPM_CUDA(cudaMemcpy(bb.data(), t.box_beg.p, sizeof(int) * nb, cudaMemcpyDeviceToHost));
  HPM_CUDA(cudaMemcpy(be.data(), t.box_end.p, sizeof(int) * nb, cudaMemcpyDeviceToHost));
  HPM_CUDA(cudaMemcpy(bp.data(), t.box_parent.p, sizeof(int) * nb, cudaMemcpyDeviceToHost));
  HPM_CUDA(cudaMemcpy(bf.data(), t.box_flags.p, nb, cudaMemcpyDeviceToHost));
  HPM_CUDA(cudaMemcpy(bc.data(), t.box_child.p, sizeof(int) * 8 * nb, cudaMemcpyDeviceToHost));
  HPM_CUDA(cudaMemcpy(bn.data(), t.box_nb.p, sizeof(int) * 27 * nb, cudaMemcpyDeviceToHost));
  int64_t c = 0, ti = 0, li = 0;
  for (int l = 0; l <= plan->max_depth; ++l) {
    for (int64_t b = plan->lvl_off[l]; b < plan->lvl_off[l + 1]; ++b) {
      if (!(bf[b] & kReal)) continue;
      if (level) level[c] = l;
      if (key) key[c] = bk[b];
      if (begin) begin[c] = bb[b];
      if (end) end[c] = be[b];
      if (leaf) leaf[c] = (bf[b] & kLeaf) ? 1 : 0;
      ++c;
      if (l >= 2) {
        if (iz) {
          const int o = (int)(bk[b] & 7u);
          const int tp[3] = {2 + (o & 1), 2 + ((o >> 1) & 1), 2 + ((o >> 2) & 1)};
          uint64_t w[4] = {0, 0, 0, 0};
          const int p = bp[b];
          for (int j = 0; j < 216; ++j) {
            const int x = j % 6, y = (j / 6) % 6, z = j / 36;
            if (std::max(std::abs(x - tp[0]), std::max(std::abs(y - tp[1]), std::abs(z - tp[2]))) < 2) continue;
            const int q = bn[(int64_t)p * 27 + (x >> 1) + 3 * (y >> 1) + 9 * (z >> 1)];
            if (q < 0) continue;
            if (bc[(int64_t)q * 8 + (x & 1) + 2 * (y & 1) + 4 * (z & 1)] < 0) continue;
            w[j / 64] |= 1ull << (j % 64);
          }
          for (int k = 0; k < 4; ++k) iz[ti * 4 + k] = w[k];
        }
        ++ti;
      }
      if (bf[b] & kLeaf) {
        if (near) {
          uint32_t m = 0;
          for (int k = 0; k < 27; ++k)
            if (bn[b * 27 + k] >= 0) m |= 1u << k;
          near[li] = m;
        }
        ++li;
      }
    }
  }
  if (perm) {
    std::vector<uint32_t> pm(n);
    HPM_CUDA(cudaMemcpy(pm.data(), t.perm.p, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < n; ++i) perm[i] = pm[i];
  }
  return HPM_OK;
}

hpm_status hpm_get_boxes(hpm_plan_t plan, int32_t *level, uint64_t *key, uint8_t *flags) {
  if (!plan) return HPM_ERR_INVALID_ARG;
  if (!plan->built) return HPM_ERR_NOT_BUILT;
  HPM_CUDA(cudaDeviceSynchronize());
  const int64_t nb = plan->nbox;
  if (nb == 0) return HPM_OK;
  if (key) HPM_CUDA(cudaMemcpy(key, plan->t.box_key.p, sizeof(uint64_t) * nb, cudaMemcpyDeviceToHost));
  if (flags) {
    std::vector<uint8_t> f(nb);
    HPM_CUDA(cudaMemcpy(f.data(), plan->t.box_flags.p, nb, cudaMemcpyDeviceToHost));
    for (int64_t b = 0; b < nb; ++b)
      flags[b] = ((f[b] & kReal) ? 1 : 0) | ((f[b] & kInternal) ? 2 : 0) | ((f[b] & kLeaf) ? 4 : 0);
  }
  if (level)
    for (int l = 0; l <= plan->max_depth; ++l)
      for (int64_t b = plan->lvl_off[l]; b < plan->lvl_off[l + 1]; ++b) level[b] = l;
  return HPM_OK;
}

hpm_status hpm_get_stage(hpm_plan_t plan, int stage, float *h_out, int64_t count) {
  if (!plan || !h_out) return HPM_ERR_INVALID_ARG;
  if (!plan->built) return HPM_ERR_NOT_BUILT;
  const int64_t m3 = (int64_t)plan->ng * plan->ng * plan->ng;
  HPM_CUDA(cudaDeviceSynchronize());
  if (plan->n == 0) return HPM_OK;
  if (stage == HPM_STAGE_MASSES) {
    const int64_t off2 = plan->max_depth >= 2 ? plan->lvl_off[2] : plan->nbox;
    const int64_t rows = plan->nbox - off2;
    if (count < rows * m3) return HPM_ERR_INVALID_ARG;
    if (rows) HPM_CUDA(cudaMemcpy(h_out, plan->s.grid.p, sizeof(float) * rows * m3, cudaMemcpyDeviceToHost));
    return HPM_OK;
  }
  if (stage == HPM_STAGE_M2L || stage == HPM_STAGE_LOCAL) {
    const int64_t nt = plan->ntgt;
    const int64_t m3 = (int64_t)plan->ng_loc * plan->ng_loc * plan->ng_loc;  // target gridlet
    if (count < nt * (m3 + 1)) return HPM_ERR_INVALID_ARG;
    if (!nt) return HPM_OK;
    const DevBuf &v = stage == HPM_STAGE_M2L ? plan->s.m2l_raw : plan->s.loc;
    const DevBuf &c = stage == HPM_STAGE_M2L ? plan->s.m2lc : plan->s.locc;
    HPM_CUDA(cudaMemcpy(h_out, v.p, sizeof(float) * nt * m3, cudaMemcpyDeviceToHost));
    HPM_CUDA(cudaMemcpy(h_out + nt * m3, c.p, sizeof(float) * nt, cudaMemcpyDeviceToHost));
    return HPM_OK;
  }
  return HPM_ERR_INVALID_ARG;
}

hpm_status hpm_get_stats(hpm_plan_t plan, hpm_stats *st) {
  if (!plan || !st) return HPM_ERR_INVALID_ARG;
  *st = plan->stats;
  plan_bytes(plan, &st->table_bytes, &st->work_bytes);
  if (plan->events_ready) {
    HPM_CUDA(cudaEventSynchronize(plan->ev[7]));
    float v[8] = {0};
    for (int i = 0; i < 7; ++i) cudaEventElapsedTime(&v[i], plan->ev[i], plan->ev[i + 1]);
    float tree = 0.f, tot = 0.f;
    cudaEventElapsedTime(&tree, plan->ev[8], plan->ev[9]);
    cudaEventElapsedTime(&tot, plan->ev[0], plan->ev[7]);
    cudaGetLastError();
    HPM_TRY(take_solve_error(plan, 0));
    st->ms_tree = tree;
    st->ms_p2g = v[0] + v[1];
    st->ms_m2m = v[2];
    st->ms_m2l = v[3];
    st->ms_l2l = v[4];
    st->ms_g2p = v[5];
    st->ms_p2p = v[6];
    st->ms_total = tot + tree;
    float mk = 0.f;
    if (plan->stats.m2l_parents > 0 && cudaEventElapsedTime(&mk, plan->ev[10], plan->ev[11]) == cudaSuccess)
      st->ms_m2l_kernel = mk;
    cudaGetLastError();
  }
  return HPM_OK;
}

hpm_status hpm_destroy(hpm_plan_t plan) {
  if (!plan) return HPM_OK;
  cudaDeviceSynchronize();
  release_all(plan, 0);
  cudaStreamSynchronize(0);
  for (auto &ev : plan->ev)
    if (ev) cudaEventDestroy(ev);
  for (auto &ev : plan->io_ev)
    if (ev) cudaEventDestroy(ev);
  if (plan->io_stream) cudaStreamDestroy(plan->io_stream);
  if (plan->h_pin) cudaFreeHost(plan->h_pin);
  cudaGetLastError();
  delete plan;
  return HPM_OK;
}

}  // extern "C"
