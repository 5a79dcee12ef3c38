// C ABI entry points: context, drop set-up, transforms and operator evaluation.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <set>

#include "internal.h"

namespace shbim {

int fail(shbim_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return code;
}

int cuda_fail(shbim_ctx* ctx, cudaError_t e, const char* what) {
  if (ctx) ctx->err = std::string(what) + ": " + cudaGetErrorString(e);
  return SHBIM_ERR_CUDA;
}

int pairs_tile_targets();

// Shape-dependent state for the current layout: drop centres (x_00 / sqrt(4 pi), the mean
// position over the parameter sphere), the device drop table, geometry and singular rows.
int rebuild_geometry(shbim_ctx* ctx, const double* xcoef_dev, cudaStream_t s) {
  SHBIM_CUDA(ctx, cudaStreamSynchronize(s));
  ctx->geom_version++;  // invalidates captured operator graphs
  ctx->xcoef_cur = xcoef_dev;
  for (auto& d : ctx->drops) {
    double c00[3];
    for (int c = 0; c < 3; ++c)
      SHBIM_CUDA(ctx, cudaMemcpy(&c00[c], xcoef_dev + 3 * d.coef_off + (int64_t)c * d.nc, sizeof(double),
                                 cudaMemcpyDeviceToHost));
    for (int c = 0; c < 3; ++c) d.centre[c] = c00[c] / std::sqrt(4.0 * kPi);
  }
  std::vector<DropDev> dd(ctx->n_drops);
  for (int i = 0; i < ctx->n_drops; ++i) {
    const Drop& d = ctx->drops[i];
    dd[i] = DropDev{d.p, d.q, d.nt, d.ns, d.nc, d.coef_off, d.tgt_off, d.src_off, d.lam,
                    d.centre[0], d.centre[1], d.centre[2], d.rows_lap, d.rows_sto};
  }
  SHBIM_CUDA(ctx, cudaMemcpy(ctx->drops_dev, dd.data(), dd.size() * sizeof(DropDev), cudaMemcpyHostToDevice));
  int rc;
  if ((rc = build_geometry(ctx, xcoef_dev, s))) return rc;
  if ((rc = build_quantized_sources(ctx, s))) return rc;
  if ((rc = build_stokes_preconditioner(ctx, xcoef_dev, s))) return rc;
  if ((rc = ctx->rows_prec == SHBIM_PREC_DF64 ? build_singular_rows_df(ctx, s, xcoef_dev)
                                              : build_singular_rows(ctx, xcoef_dev, s)))
    return rc;
  if ((rc = build_near(ctx, xcoef_dev, s))) return rc;
  return SHBIM_OK;
}

namespace {

void free_drop_state(shbim_ctx* ctx) {
  for (auto& d : ctx->drops) {
    cudaFree(d.rows_lap);
    cudaFree(d.rows_sto);
  }
  ctx->drops.clear();
  cudaFree(ctx->geo.tgt);
  cudaFree(ctx->geo.src);
  cudaFree(ctx->geo.tgt32);
  cudaFree(ctx->geo.src32);
  cudaFree(ctx->geo.src32lo);
  cudaFree(ctx->geo.srcq);
  cudaFree(ctx->geo.tgt_drop);
  ctx->geo = Geometry{};
  cudaFree(ctx->tiles_dev);
  ctx->tiles_dev = nullptr;
  cudaFree(ctx->drops_dev);
  ctx->drops_dev = nullptr;
  cudaFree(ctx->lamm1_dev);
  ctx->lamm1_dev = nullptr;
  cudaFree(ctx->prec_basis);
  cudaFree(ctx->prec_dots);
  cudaFree(ctx->prec_fac);
  ctx->prec_basis = ctx->prec_dots = ctx->prec_fac = nullptr;
  cudaFree(ctx->dens_up);
  ctx->dens_up = nullptr;
  cudaFree(ctx->dens_up32);
  ctx->dens_up32 = nullptr;
  cudaFree(ctx->dens_up32lo);
  ctx->dens_up32lo = nullptr;
  cudaFree(ctx->part);
  ctx->part = nullptr;
  cudaFree(ctx->grid_out);
  ctx->grid_out = nullptr;
  cudaFree(ctx->xup);
  ctx->xup = nullptr;
  ctx->tiles.clear();
  for (auto& g : ctx->groups) {
    cudaFree(g.idx);
    cudaFree(g.coef);
    cudaFree(g.src);
    cudaFree(g.tgt);
    cudaFree(g.tgt3);
  }
  ctx->groups.clear();
  ctx->n_drops = 0;
  ctx->ncoef = ctx->ntarget = ctx->nsource = 0;
}

template <typename T>
int dalloc(shbim_ctx* ctx, T** p, size_t n, const char* what) {
  if (cudaMalloc((void**)p, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) {
    *p = nullptr;
    return fail(ctx, SHBIM_ERR_NOMEM, std::string("cudaMalloc ") + what);
  }
  return SHBIM_OK;
}

bool valid_opts(const shbim_opts& o) {
  return (o.precision == SHBIM_PREC_FP64 || o.precision == SHBIM_PREC_FP32_COMP ||
          o.precision == SHBIM_PREC_DF64) &&
         o.gmres_restart >= 1 && o.gmres_restart <= 200 && o.gmres_tol > 0.0 && o.gmres_tol < 1.0 &&
         o.gmres_maxiter >= 1 && std::isfinite(o.R) && o.R > 0.0;
}

}  // namespace
}  // namespace shbim

using namespace shbim;

extern "C" {

int shbim_create(const shbim_opts* opts, shbim_ctx** out) {
  if (!out) return SHBIM_ERR_ARG;
  *out = nullptr;
  shbim_opts o{};
  o.precision = SHBIM_PREC_FP64;
  o.gmres_restart = 50;
  o.gmres_tol = 1e-8;
  o.gmres_maxiter = 1000;
  o.R = 1.0;
  if (opts) {
    o = *opts;
    if (o.gmres_restart == 0) o.gmres_restart = 50;
    if (o.gmres_tol == 0.0) o.gmres_tol = 1e-8;
    if (o.gmres_maxiter == 0) o.gmres_maxiter = 1000;
  }
  if (!valid_opts(o)) return SHBIM_ERR_ARG;
  shbim_ctx* ctx = new shbim_ctx();
  ctx->opts = o;
  *out = ctx;
  return SHBIM_OK;
}

int shbim_destroy(shbim_ctx* ctx) {
  if (!ctx) return SHBIM_ERR_ARG;
  cudaDeviceSynchronize();
  free_drop_state(ctx);
  for (auto& kv : ctx->tables) free_degree_tables(kv.second);
  cudaFree(ctx->sht_scratch);
  cudaFree(ctx->dq_ext_dev);
  cudaFree(ctx->dq_far);
  cudaFree(ctx->rot_coef);
  cudaFree(ctx->wbuf);
  cudaFree(ctx->vbuf);
  cudaFree(ctx->gm.V);
  cudaFree(ctx->gm.w);
  cudaFree(ctx->gm.x);
  cudaFree(ctx->gm.b);
  cudaFree(ctx->gm.h);
  cudaFree(ctx->gm.Av);
  cudaFree(ctx->gm.diag);
  cudaFree(ctx->gm.tmp);
  cudaFree(ctx->gm.y);
  {
    auto& N = ctx->near;
    cudaFree(N.stats); cudaFree(N.det_t); cudaFree(N.det_j); cudaFree(N.pair_t); cudaFree(N.pair_j);
    cudaFree(N.fgeo); cudaFree(N.fgeo32); cudaFree(N.fstr); cudaFree(N.fstr32); cudaFree(N.foff_dev);
    cudaFree(N.fgeo32lo); cudaFree(N.fstr32lo); cudaFree(N.groups);
    for (auto& g : N.groups_d) {
      cudaFree(g.idx); cudaFree(g.coef); cudaFree(g.fine);
    }
  }
  for (auto& g : ctx->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    cudaFree(g.in);
    cudaFree(g.out);
  }
  for (auto& c : ctx->cycles)
    if (c.exec) cudaGraphExecDestroy(c.exec);
  cudaFree(ctx->gm.dstate);
  cudaFree(ctx->gm.istate);
  cudaFree(ctx->gm.vstage);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  cudaFree(ctx->pair_queue);
  if (ctx->side) cudaStreamDestroy(ctx->side);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_coarse) cudaEventDestroy(ctx->ev_coarse);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  cudaFree(ctx->phys.buf);
  cudaFree(ctx->phys.grid);
  cudaFree(ctx->phys.state);
  cudaFree(ctx->phys.lb);
  cudaFree(ctx->phys.feat);
  cudaFree(ctx->phys.guess);
  cudaFree(ctx->phys.rep);
  cudaFree(ctx->dens_split);
  for (auto& L : ctx->lanes) {
    cudaFree(L.rot);
    cudaFree(L.w);
    cudaFree(L.v);
    cudaFree(L.F);
    cudaFree(L.xdf);
    cudaFree(L.rexp);
  }
  cudaFree(ctx->tc_err);
  cudaFree(ctx->gm.xr);
  cudaFree(ctx->gm.rr);
  cudaFree(ctx->gm.dr);
  if (ctx->gm.h_host) cudaFreeHost(ctx->gm.h_host);
  delete ctx;
  return SHBIM_OK;
}

const char* shbim_last_error(shbim_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int shbim_set_precision(shbim_ctx* ctx, int precision) {
  if (!ctx) return SHBIM_ERR_ARG;
  if (precision != SHBIM_PREC_FP64 && precision != SHBIM_PREC_FP32_COMP && precision != SHBIM_PREC_DF64)
    return fail(ctx, SHBIM_ERR_ARG, "precision must be SHBIM_PREC_FP64, SHBIM_PREC_FP32_COMP or SHBIM_PREC_DF64");
  ctx->opts.precision = precision;
  return SHBIM_OK;
}

int shbim_set_R(shbim_ctx* ctx, double R) {
  if (!ctx) return SHBIM_ERR_ARG;
  if (!(R > 0.0) || !std::isfinite(R)) return fail(ctx, SHBIM_ERR_ARG, "R must be positive");
  if (R != ctx->opts.R) ctx->geom_version++;  // the electric system's factor is captured in graphs
  ctx->opts.R = R;
  return SHBIM_OK;
}

int64_t shbim_launch_count(shbim_ctx* ctx) { return ctx ? ctx->launches : -1; }

int shbim_set_wait_limit(shbim_ctx* ctx, double seconds) {
  if (!ctx) return SHBIM_ERR_ARG;
  if (!(seconds >= 1e-3 && seconds <= 60.0)) return fail(ctx, SHBIM_ERR_ARG, "wait limit must be in [1e-3, 60] s");
  ctx->wait_ns = (uint64_t)(seconds * 1e9);
  ctx->geom_version++;  // captured graphs hold the old limit as a kernel argument
  return SHBIM_OK;
}

int64_t shbim_operator_applications(shbim_ctx* ctx) { return ctx ? ctx->applications : -1; }

int shbim_set_rows_precision(shbim_ctx* ctx, int precision) {
  if (!ctx) return SHBIM_ERR_ARG;
  if (precision != SHBIM_PREC_FP64 && precision != SHBIM_PREC_DF64)
    return fail(ctx, SHBIM_ERR_ARG, "row precision must be SHBIM_PREC_FP64 or SHBIM_PREC_DF64");
  ctx->rows_prec = precision;
  return SHBIM_OK;
}

int shbim_set_self_precision(shbim_ctx* ctx, int precision) {
  if (!ctx) return SHBIM_ERR_ARG;
  if (precision != SHBIM_PREC_FP32_COMP && precision != SHBIM_PREC_DF64)
    return fail(ctx, SHBIM_ERR_ARG, "self-row precision must be SHBIM_PREC_FP32_COMP or SHBIM_PREC_DF64");
  if (precision != ctx->self_prec) ctx->geom_version++;  // captured graphs hold the other kernel
  ctx->self_prec = precision;
  return SHBIM_OK;
}

int shbim_set_tensor_cores(shbim_ctx* ctx, int mask) {
  if (!ctx) return SHBIM_ERR_ARG;
  if (mask & ~SHBIM_TC_ALL) return fail(ctx, SHBIM_ERR_ARG, "unknown tensor-core stage bit");
  ctx->tc_rows = (mask & SHBIM_TC_FOURIER) != 0;
  ctx->tc_rot = (mask & SHBIM_TC_ROTATION) != 0;
  ctx->tc_leg = (mask & SHBIM_TC_LEGENDRE) != 0;
  return SHBIM_OK;
}

int shbim_set_autotune(shbim_ctx* ctx, int on) {
  if (!ctx) return SHBIM_ERR_ARG;
  ctx->autotune = on != 0;
  for (auto& c : ctx->pair_cfg) c = shbim_ctx::PairCfg{1, ctx->pair_splits, !ctx->autotune};
  ctx->geom_version++;  // captured graphs hold the old launch shapes
  return SHBIM_OK;
}

int shbim_pair_shape(shbim_ctx* ctx, int kind, int* tpt_host, int* splits_host) {
  if (!ctx) return SHBIM_ERR_ARG;
  if (kind < 0 || kind > 4) return fail(ctx, SHBIM_ERR_ARG, "kind must be 0 (Laplace DL), 1 (SL), 2 (Stokes S + D), 3 (S) or 4 (D)");
  if (tpt_host) *tpt_host = ctx->pair_cfg[kind].tpt;
  if (splits_host) *splits_host = ctx->pair_cfg[kind].splits;
  return ctx->pair_cfg[kind].tuned ? 1 : 0;
}

int shbim_set_pair_shape(shbim_ctx* ctx, int kind, int tpt, int splits) {
  if (!ctx) return SHBIM_ERR_ARG;
  if (ctx->n_drops == 0) return fail(ctx, SHBIM_ERR_ARG, "no drops set");
  if (kind < 0 || kind > 4) return fail(ctx, SHBIM_ERR_ARG, "kind must be 0 (Laplace DL), 1 (SL), 2 (Stokes S + D), 3 (S) or 4 (D)");
  if (tpt != 1 && tpt != 2 && tpt != 4) return fail(ctx, SHBIM_ERR_ARG, "targets per thread must be 1, 2 or 4");
  if (splits < 1 || splits > ctx->split_max) return fail(ctx, SHBIM_ERR_ARG, "split count out of range");
  ctx->pair_cfg[kind] = shbim_ctx::PairCfg{tpt, splits, true, ctx->pair_cfg[kind].queue};
  ctx->geom_version++;
  return SHBIM_OK;
}

int shbim_pair_queue(shbim_ctx* ctx, int kind) {
  if (!ctx) return SHBIM_ERR_ARG;
  if (kind < 0 || kind > 4) return fail(ctx, SHBIM_ERR_ARG, "kind must be 0 (Laplace DL), 1 (SL), 2 (Stokes S + D), 3 (S) or 4 (D)");
  return ctx->pair_cfg[kind].queue ? 1 : 0;
}

int shbim_set_pair_queue(shbim_ctx* ctx, int kind, int on) {
  if (!ctx) return SHBIM_ERR_ARG;
  if (ctx->n_drops == 0) return fail(ctx, SHBIM_ERR_ARG, "no drops set");
  if (kind < 0 || kind > 4) return fail(ctx, SHBIM_ERR_ARG, "kind must be 0 (Laplace DL), 1 (SL), 2 (Stokes S + D), 3 (S) or 4 (D)");
  ctx->pair_cfg[kind].queue = on != 0;
  ctx->pair_cfg[kind].tuned = true;
  ctx->geom_version++;
  return SHBIM_OK;
}

int shbim_set_graphs(shbim_ctx* ctx, int on) {
  if (!ctx) return SHBIM_ERR_ARG;
  ctx->graphs_on = on != 0;
  return SHBIM_OK;
}

int shbim_set_concurrency(shbim_ctx* ctx, int on) {
  if (!ctx) return SHBIM_ERR_ARG;
  ctx->concurrent = on != 0;
  ctx->geom_version++;  // captured operator graphs have the other stream layout
  return SHBIM_OK;
}

int shbim_sizes(shbim_ctx* ctx, int64_t* nc, int64_t* nt, int64_t* ns) {
  if (!ctx) return SHBIM_ERR_ARG;
  if (nc) *nc = ctx->ncoef;
  if (nt) *nt = ctx->ntarget;
  if (ns) *ns = ctx->nsource;
  return SHBIM_OK;
}

int shbim_set_drops(shbim_ctx* ctx, int n_drops, const int32_t* p_host, const double* lambda_host,
                    const double* xcoef_dev, void* stream) {
  if (!ctx) return SHBIM_ERR_ARG;
  if (n_drops < 1 || !p_host || !xcoef_dev) return fail(ctx, SHBIM_ERR_ARG, "need n_drops >= 1, p and x");
  for (int i = 0; i < n_drops; ++i) {
    if (p_host[i] < 1 || p_host[i] > 64) return fail(ctx, SHBIM_ERR_ARG, "degree p must be in [1, 64]");
    if (lambda_host && (!std::isfinite(lambda_host[i]) || lambda_host[i] <= 0.0))
      return fail(ctx, SHBIM_ERR_ARG, "viscosity ratios must be positive");
  }
  cudaStream_t s = (cudaStream_t)stream;
  SHBIM_CUDA(ctx, cudaStreamSynchronize(s));
  bool same = ctx->n_drops == n_drops;
  for (int i = 0; same && i < n_drops; ++i) same = ctx->drops[i].p == p_host[i];
  if (same) {
    // same layout: keep every allocation, refresh the shape-dependent state only
    std::vector<double> lm1(n_drops);
    for (int i = 0; i < n_drops; ++i) {
      ctx->drops[i].lam = lambda_host ? lambda_host[i] : 1.0;
      lm1[i] = ctx->drops[i].lam - 1.0;
    }
    SHBIM_CUDA(ctx, cudaMemcpy(ctx->lamm1_dev, lm1.data(), n_drops * sizeof(double), cudaMemcpyHostToDevice));
    return rebuild_geometry(ctx, xcoef_dev, s);
  }
  free_drop_state(ctx);
  int rc;
  // tables per distinct degree (kept across calls)
  for (int i = 0; i < n_drops; ++i) {
    const int p = p_host[i];
    if (!ctx->tables.count(p)) {
      DegreeTables* T = nullptr;
      if ((rc = build_degree_tables(ctx, p, &T))) return rc;
      ctx->tables[p] = T;
    }
  }
  // layout
  ctx->drops.resize(n_drops);
  int64_t co = 0, to = 0, so = 0;
  for (int i = 0; i < n_drops; ++i) {
    Drop& d = ctx->drops[i];
    d.p = p_host[i];
    d.q = 2 * d.p + 1;
    d.nc = ncoef(d.p);
    d.nt = npts(d.p);
    d.ns = npts(d.q);
    d.coef_off = co;
    d.tgt_off = to;
    d.src_off = so;
    d.lam = lambda_host ? lambda_host[i] : 1.0;
    d.tab = ctx->tables[d.p];
    co += d.nc;
    to += d.nt;
    so += d.ns;
  }
  ctx->n_drops = n_drops;
  ctx->ncoef = co;
  ctx->ntarget = to;
  ctx->nsource = so;
  // geometry and workspaces
  if ((rc = dalloc(ctx, &ctx->geo.tgt, 7 * (size_t)to, "targets")) ||
      (rc = dalloc(ctx, &ctx->geo.src, 7 * (size_t)so, "sources")) ||
      (rc = dalloc(ctx, &ctx->geo.tgt32, 7 * (size_t)to, "targets32")) ||
      (rc = dalloc(ctx, &ctx->geo.src32, 7 * (size_t)so, "sources32")) ||
      (rc = dalloc(ctx, &ctx->geo.src32lo, 7 * (size_t)so, "sources32 low parts")) ||
      (rc = dalloc(ctx, &ctx->geo.srcq, 6 * (size_t)so, "quantised source positions")) ||
      (rc = dalloc(ctx, &ctx->geo.tgt_drop, (size_t)to, "target drop ids")) ||
      (rc = dalloc(ctx, &ctx->dens_up, 6 * (size_t)so, "source strengths")) ||
      (rc = dalloc(ctx, &ctx->dens_up32, 6 * (size_t)so, "source strengths32")) ||
      (rc = dalloc(ctx, &ctx->dens_up32lo, 6 * (size_t)so, "source strengths32 low parts")) ||
      (rc = dalloc(ctx, &ctx->grid_out, 3 * (size_t)to, "target values")) ||
      (rc = dalloc(ctx, &ctx->xup, 3 * (size_t)kNumTab * so, "position derivatives")))
    return rc;
  for (auto& d : ctx->drops) {
    if ((rc = dalloc(ctx, &d.rows_lap, 2 * (size_t)d.nt * kNumLap * d.nc, "laplace rows")) ||
        (rc = dalloc(ctx, &d.rows_sto, 2 * (size_t)d.nt * kNumSto * d.nc, "stokes rows")))
      return rc;
  }
  // drops grouped by degree: the transforms of an operator application take one launch per degree
  {
    std::vector<int> order;
    for (int i = 0; i < n_drops; ++i) {
      bool seen = false;
      for (int k : order) seen = seen || ctx->drops[k].p == ctx->drops[i].p;
      if (!seen) order.push_back(i);
    }
    for (int first : order) {
      std::vector<int> idx;
      std::vector<int64_t> co, sr, tg, tg3;
      for (int i = 0; i < n_drops; ++i)
        if (ctx->drops[i].p == ctx->drops[first].p) {
          idx.push_back(i);
          co.push_back(ctx->drops[i].coef_off);
          sr.push_back(ctx->drops[i].src_off);
          tg.push_back(ctx->drops[i].tgt_off);
          tg3.push_back(3 * ctx->drops[i].tgt_off);
        }
      DegreeGroup G;
      G.tab = ctx->drops[first].tab;
      G.n = (int)idx.size();
      G.first = first;
      ctx->groups.push_back(G);
      DegreeGroup& g = ctx->groups.back();
      if ((rc = dalloc(ctx, &g.idx, idx.size(), "degree group")) || (rc = dalloc(ctx, &g.coef, co.size(), "degree group")) ||
          (rc = dalloc(ctx, &g.src, sr.size(), "degree group")) || (rc = dalloc(ctx, &g.tgt, tg.size(), "degree group")) ||
          (rc = dalloc(ctx, &g.tgt3, tg3.size(), "degree group")))
        return rc;
      SHBIM_CUDA(ctx, cudaMemcpy(g.tgt3, tg3.data(), tg3.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
      SHBIM_CUDA(ctx, cudaMemcpy(g.idx, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice));
      SHBIM_CUDA(ctx, cudaMemcpy(g.coef, co.data(), co.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
      SHBIM_CUDA(ctx, cudaMemcpy(g.src, sr.data(), sr.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
      SHBIM_CUDA(ctx, cudaMemcpy(g.tgt, tg.data(), tg.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
    }
  }
  {
    std::vector<int> tdrop(to);
    for (int i = 0; i < n_drops; ++i)
      std::fill(tdrop.begin() + ctx->drops[i].tgt_off,
                tdrop.begin() + ctx->drops[i].tgt_off + ctx->drops[i].nt, i);
    SHBIM_CUDA(ctx, cudaMemcpy(ctx->geo.tgt_drop, tdrop.data(), to * sizeof(int), cudaMemcpyHostToDevice));
    if ((rc = dalloc(ctx, &ctx->drops_dev, n_drops, "drop table"))) return rc;
    std::vector<double> lm1(n_drops);
    for (int i = 0; i < n_drops; ++i) lm1[i] = ctx->drops[i].lam - 1.0;
    if ((rc = dalloc(ctx, &ctx->lamm1_dev, n_drops, "viscosity contrasts"))) return rc;
    SHBIM_CUDA(ctx, cudaMemcpy(ctx->lamm1_dev, lm1.data(), n_drops * sizeof(double), cudaMemcpyHostToDevice));
  }
  // all-pairs tiling: tiles never cross a drop; sources split so that the grid fills the GPU
  {
    const int TT = pairs_tile_targets();
    int64_t min_other = so;
    for (int i = 0; i < n_drops; ++i) {
      const Drop& d = ctx->drops[i];
      for (int t0 = 0; t0 < d.nt; t0 += TT)
        ctx->tiles.push_back(PairTile{i, (int)(d.tgt_off + t0), std::min(TT, d.nt - t0)});
      min_other = std::min<int64_t>(min_other, so - d.ns);
    }
    // largest work first (targets x other drops' sources): the grid's first CTAs and the
    // persistent form's first units take the longest tiles
    std::stable_sort(ctx->tiles.begin(), ctx->tiles.end(), [&](const PairTile& a, const PairTile& b) {
      return (int64_t)a.nt * (so - ctx->drops[a.drop].ns) > (int64_t)b.nt * (so - ctx->drops[b.drop].ns);
    });
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    // about 8 CTAs per SM at 2 targets per thread (2 CTAs per tile)
    const int64_t want = (int64_t)nsm * 8;
    const int64_t ctas = 2 * (int64_t)ctx->tiles.size();
    int64_t splits = (want + ctas - 1) / ctas;
    splits = std::min<int64_t>(splits, std::max<int64_t>(1, min_other / 128));
    ctx->pair_splits = (int)std::max<int64_t>(1, std::min<int64_t>(splits, 256));
    if ((rc = dalloc(ctx, &ctx->tiles_dev, ctx->tiles.size(), "tiles"))) return rc;
    SHBIM_CUDA(ctx, cudaMemcpy(ctx->tiles_dev, ctx->tiles.data(), ctx->tiles.size() * sizeof(PairTile),
                               cudaMemcpyHostToDevice));
    ctx->cross_pairs = 0;
    for (const Drop& d : ctx->drops) ctx->cross_pairs += (int64_t)d.nt * (so - d.ns);
    ctx->split_max = (int)std::max<int64_t>(1, std::min<int64_t>(4 * splits, std::max<int64_t>(1, min_other / 64)));
    ctx->split_max = std::min(ctx->split_max, 256);
    ctx->pair_splits = std::min(ctx->pair_splits, ctx->split_max);
    for (auto& c : ctx->pair_cfg) c = shbim_ctx::PairCfg{1, ctx->pair_splits, !ctx->autotune};
    if ((rc = dalloc(ctx, &ctx->part, (size_t)ctx->split_max * 3 * to, "pair partials"))) return rc;
    if (!ctx->pair_queue) {
      if ((rc = dalloc(ctx, &ctx->pair_queue, 2, "pair work counter"))) return rc;
      SHBIM_CUDA(ctx, cudaMemset(ctx->pair_queue, 0, 2 * sizeof(int)));
    }
  }
  return rebuild_geometry(ctx, xcoef_dev, s);
}

int shbim_target_geometry(shbim_ctx* ctx, double* out_dev, void* stream) {
  if (!ctx || !out_dev) return SHBIM_ERR_ARG;
  if (ctx->n_drops == 0) return fail(ctx, SHBIM_ERR_ARG, "no drops set");
  SHBIM_CUDA(ctx, cudaMemcpyAsync(out_dev, ctx->geo.tgt, 7 * ctx->ntarget * sizeof(double),
                                  cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return SHBIM_OK;
}

int shbim_sht(shbim_ctx* ctx, int dir, int grid, int n_fields, const int32_t* field_drop_host,
              const double* in_dev, double* out_dev, void* stream) {
  if (!ctx) return SHBIM_ERR_ARG;
  if (ctx->n_drops == 0) return fail(ctx, SHBIM_ERR_ARG, "no drops set");
  if (n_fields < 0 || (n_fields > 0 && (!field_drop_host || !in_dev || !out_dev)))
    return fail(ctx, SHBIM_ERR_ARG, "bad fields or pointers");
  if (grid != SHBIM_GRID_BASE && grid != SHBIM_GRID_UP) return fail(ctx, SHBIM_ERR_ARG, "bad grid");
  if (dir != SHBIM_SHT_INVERSE && dir != SHBIM_SHT_FORWARD) return fail(ctx, SHBIM_ERR_ARG, "bad direction");
  for (int f = 0; f < n_fields; ++f)
    if (field_drop_host[f] < 0 || field_drop_host[f] >= ctx->n_drops)
      return fail(ctx, SHBIM_ERR_ARG, "field_drop: drop index out of range");
  cudaStream_t s = (cudaStream_t)stream;
  // fields are concatenated, each with its own drop's coefficient count and grid size; a run of
  // consecutive fields of one drop is one transform launch
  int64_t in_off = 0, out_off = 0;
  for (int f = 0, g; f < n_fields; f = g) {
    g = f + 1;
    while (g < n_fields && field_drop_host[g] == field_drop_host[f]) ++g;
    const Drop& d = ctx->drops[field_drop_host[f]];
    const GridTables& T = grid == SHBIM_GRID_BASE ? d.tab->base : d.tab->up;
    const int64_t n = npts(T.q);
    const int nf = g - f;
    int rc;
    if (dir == SHBIM_SHT_INVERSE) {
      rc = sht_synth(ctx, T, nf, in_dev + in_off, d.nc, 1, out_dev + out_off, n, 0, nullptr, nullptr, s);
      in_off += (int64_t)nf * d.nc;
      out_off += (int64_t)nf * n;
    } else {
      rc = sht_analysis(ctx, T, nf, in_dev + in_off, n, true, out_dev + out_off, d.nc, s);
      in_off += (int64_t)nf * n;
      out_off += (int64_t)nf * d.nc;
    }
    if (rc) return rc;
  }
  return SHBIM_OK;
}

}  // extern "C"

namespace shbim {
namespace {

}  // namespace

int ensure_side_stream(shbim_ctx* ctx) {
  if (ctx->side) return SHBIM_OK;
  if (cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_coarse, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess)
    return cuda_fail(ctx, cudaGetLastError(), "side stream");
  return SHBIM_OK;
}

namespace {

// Streams of one operator application. With two or more drops and concurrency on, the self rows
// (which overwrite the output values) and then the near-field correction (which adds into them)
// run on the library's side stream while the caller's stream synthesises the strengths and runs
// the all-pairs sums; `coarse` marks the strengths as ready for the near-field sums and `join`
// the side branch as done, before the pair partials are added into the output.
struct Branches {
  cudaStream_t side = nullptr;
  cudaEvent_t coarse = nullptr, join = nullptr;
};

// timing class of the all-pairs sums at the context's precision
int pair_class(const shbim_ctx* ctx) {
  return ctx->opts.precision == SHBIM_PREC_FP32_COMP ? SHBIM_K_PAIRS : SHBIM_K_PAIRS_FP64CLASS;
}

int fork_branches(shbim_ctx* ctx, cudaStream_t s, Branches* br) {
  br->side = s;
  if (ctx->n_drops < 2 || !ctx->concurrent) return SHBIM_OK;
  if (int rc = ensure_side_stream(ctx)) return rc;
  SHBIM_CUDA(ctx, cudaEventRecord(ctx->ev_fork, s));
  SHBIM_CUDA(ctx, cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0));
  br->side = ctx->side;
  br->coarse = ctx->ev_coarse;
  br->join = ctx->ev_join;
  return SHBIM_OK;
}

}  // namespace
}  // namespace shbim

extern "C" {

int shbim_eval_electric(shbim_ctx* ctx, int which, const double* dens_dev, double* out_dev, int out_kind,
                        void* stream) {
  if (!ctx) return SHBIM_ERR_ARG;
  if (ctx->n_drops == 0) return fail(ctx, SHBIM_ERR_ARG, "no drops set");
  if (which != SHBIM_LAPLACE_DL && which != SHBIM_LAPLACE_SL) return fail(ctx, SHBIM_ERR_ARG, "bad kernel");
  if (out_kind != SHBIM_OUT_GRID && out_kind != SHBIM_OUT_COEF) return fail(ctx, SHBIM_ERR_ARG, "bad out kind");
  if (!dens_dev || !out_dev) return fail(ctx, SHBIM_ERR_ARG, "null pointer");
  cudaStream_t s = (cudaStream_t)stream;
  const bool f32 = ctx->opts.precision != SHBIM_PREC_FP64;   // FP32 copies (FP32 and double-float sums)
  const bool lo = ctx->opts.precision == SHBIM_PREC_DF64;
  int rc;
  ctx->applications++;
  double* vals = out_kind == SHBIM_OUT_GRID ? out_dev : ctx->grid_out;
  Branches br;
  if ((rc = fork_branches(ctx, s, &br))) return rc;
  {
    TimeScope ts(ctx, SHBIM_K_SELF_GEMV, br.side);
    if ((rc = apply_self_laplace(ctx, which, dens_dev, vals, br.side))) return rc;
  }
  if (ctx->n_drops > 1) {
    TimeScope ts(ctx, SHBIM_K_SHT, s);
    for (const DegreeGroup& G : ctx->groups) {
      const DropList L = G.sources();
      const int nc = ncoef(G.tab->p);
      rc = sht_synth_drops(ctx, G.tab->up, G.n, 1, dens_dev, nc, ctx->dens_up, 0, 0, ctx->geo.src + 6 * ctx->nsource,
                           1.0, nullptr, f32 ? ctx->dens_up32 : nullptr, s, lo ? ctx->dens_up32lo : nullptr, &L);
      if (rc) return rc;
    }
  }
  if (br.coarse) SHBIM_CUDA(ctx, cudaEventRecord(br.coarse, s));
  {
    TimeScope ts(ctx, SHBIM_K_NEAR, br.side);
    if ((rc = apply_near_laplace(ctx, which, dens_dev, vals, br.side, br.coarse))) return rc;
  }
  if (br.join) SHBIM_CUDA(ctx, cudaEventRecord(br.join, br.side));
  {
    TimeScope ts(ctx, pair_class(ctx), s);
    ts.work = pairs_work(ctx, which == SHBIM_LAPLACE_SL ? 1 : 0);
    if ((rc = pairs_laplace(ctx, which, vals, s, br.join))) return rc;
  }
  if (out_kind == SHBIM_OUT_COEF) {
    TimeScope ts(ctx, SHBIM_K_SHT, s);
    for (const DegreeGroup& G : ctx->groups) {
      const DropList L = G.targets();
      rc = sht_analysis(ctx, G.tab->base, G.n, vals, 0, true, out_dev, ncoef(G.tab->p), s, 1, &L);
      if (rc) return rc;
    }
  }
  return SHBIM_OK;
}

int shbim_eval_stokes(shbim_ctx* ctx, const double* f_dev, const double* u_dev, double* out_dev,
                      int out_kind, void* stream) {
  if (!ctx) return SHBIM_ERR_ARG;
  if (ctx->n_drops == 0) return fail(ctx, SHBIM_ERR_ARG, "no drops set");
  if (!f_dev && !u_dev) return fail(ctx, SHBIM_ERR_ARG, "need f or u");
  if (out_kind != SHBIM_OUT_GRID && out_kind != SHBIM_OUT_COEF) return fail(ctx, SHBIM_ERR_ARG, "bad out kind");
  if (!out_dev) return fail(ctx, SHBIM_ERR_ARG, "null output");
  cudaStream_t s = (cudaStream_t)stream;
  const bool f32 = ctx->opts.precision != SHBIM_PREC_FP64;
  const bool lo = ctx->opts.precision == SHBIM_PREC_DF64;
  const int64_t NS = ctx->nsource;
  int rc;
  ctx->applications++;
  double* vals = out_kind == SHBIM_OUT_GRID ? out_dev : ctx->grid_out;
  Branches br;
  if ((rc = fork_branches(ctx, s, &br))) return rc;
  {
    TimeScope ts(ctx, SHBIM_K_SELF_GEMV, br.side);
    if ((rc = apply_self_stokes(ctx, f_dev, u_dev, vals, br.side))) return rc;
  }
  if (ctx->n_drops > 1) {
    TimeScope ts(ctx, SHBIM_K_SHT, s);
    for (const DegreeGroup& G : ctx->groups) {
      const DropList L = G.sources();
      const int nc = ncoef(G.tab->p);
      const double* w = ctx->geo.src + 6 * NS;
      if (f_dev) {
        rc = sht_synth_drops(ctx, G.tab->up, G.n, 3, f_dev, nc, ctx->dens_up, NS, 0, w, 1.0, nullptr,
                             f32 ? ctx->dens_up32 : nullptr, s, lo ? ctx->dens_up32lo : nullptr, &L);
        if (rc) return rc;
      }
      if (u_dev) {
        // strength -6 (lambda_j - 1) u per drop
        rc = sht_synth_drops(ctx, G.tab->up, G.n, 3, u_dev, nc, ctx->dens_up + 3 * NS, NS, 0, w, -6.0, ctx->lamm1_dev,
                             f32 ? ctx->dens_up32 + 3 * NS : nullptr, s, lo ? ctx->dens_up32lo + 3 * NS : nullptr, &L);
        if (rc) return rc;
      }
    }
  }
  if (br.coarse) SHBIM_CUDA(ctx, cudaEventRecord(br.coarse, s));
  {
    TimeScope ts(ctx, SHBIM_K_NEAR, br.side);
    if ((rc = apply_near_stokes(ctx, f_dev, u_dev, vals, br.side, br.coarse))) return rc;
  }
  if (br.join) SHBIM_CUDA(ctx, cudaEventRecord(br.join, br.side));
  {
    TimeScope ts(ctx, pair_class(ctx), s);
    ts.work = pairs_work(ctx, f_dev && u_dev ? 2 : (f_dev ? 3 : 4));
    if ((rc = pairs_stokes(ctx, f_dev != nullptr, u_dev != nullptr, vals, s, br.join))) return rc;
  }
  if (out_kind == SHBIM_OUT_COEF) {
    TimeScope ts(ctx, SHBIM_K_SHT, s);
    for (const DegreeGroup& G : ctx->groups) {
      const DropList L = G.targets3();
      const int p = G.tab->p;
      rc = sht_analysis(ctx, G.tab->base, 3 * G.n, vals, npts(p), true, out_dev, ncoef(p), s, 3, &L);
      if (rc) return rc;
    }
  }
  return SHBIM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- timing and right-hand side

namespace shbim {

TimeScope::TimeScope(shbim_ctx* c, int k, cudaStream_t st) : ctx(c), cls(k), s(st) {
  if (!ctx->timing) return;
  // launches being captured into a graph are not timed (their replays run as one graph launch)
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
  cudaEvent_t a;
  if (ctx->event_pool.empty()) {
    cudaEventCreate(&a);
  } else {
    a = ctx->event_pool.back();
    ctx->event_pool.pop_back();
  }
  cudaEventRecord(a, s);
  b = a;
}

TimeScope::~TimeScope() {
  if (!ctx->timing || !b) return;
  cudaEvent_t e;
  if (ctx->event_pool.empty()) {
    cudaEventCreate(&e);
  } else {
    e = ctx->event_pool.back();
    ctx->event_pool.pop_back();
  }
  cudaEventRecord(e, s);
  ctx->timed.push_back(shbim_ctx::TimedRange{cls, b, e, work});
}

namespace {
struct FieldShape {
  double g[6];   // xx, xy, xz, yy, yz, zz
};

// scale (E_u + eq G x) . n on every target
__global__ void k_field_normal(const double* __restrict__ tgt, int64_t ntarget, double ex, double ey,
                               double ez, double eq, FieldShape G, double scale, double* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntarget) return;
  const double x = tgt[t], y = tgt[ntarget + t], z = tgt[2 * ntarget + t];
  const double nx = tgt[3 * ntarget + t], ny = tgt[4 * ntarget + t], nz = tgt[5 * ntarget + t];
  const double Ex = ex + eq * (G.g[0] * x + G.g[1] * y + G.g[2] * z);
  const double Ey = ey + eq * (G.g[1] * x + G.g[3] * y + G.g[4] * z);
  const double Ez = ez + eq * (G.g[2] * x + G.g[4] * y + G.g[5] * z);
  out[t] = scale * (Ex * nx + Ey * ny + Ez * nz);
}
}  // namespace

}  // namespace shbim

extern "C" {

int shbim_set_timing(shbim_ctx* ctx, int on) {
  if (!ctx) return SHBIM_ERR_ARG;
  SHBIM_CUDA(ctx, cudaDeviceSynchronize());
  for (auto& r : ctx->timed) {
    ctx->event_pool.push_back(r.a);
    ctx->event_pool.push_back(r.b);
  }
  ctx->timed.clear();
  for (int k = 0; k < SHBIM_K_COUNT; ++k) {
    ctx->class_ms[k] = 0.0;
    ctx->class_launches[k] = 0;
    ctx->class_work[k] = 0.0;
  }
  ctx->timing = on != 0;
  return SHBIM_OK;
}

namespace {
int collect_timing(shbim_ctx* ctx) {
  SHBIM_CUDA(ctx, cudaDeviceSynchronize());
  for (auto& r : ctx->timed) {
    float t = 0.f;
    SHBIM_CUDA(ctx, cudaEventElapsedTime(&t, r.a, r.b));
    ctx->class_ms[r.cls] += t;
    ctx->class_launches[r.cls] += 1;
    ctx->class_work[r.cls] += r.work;
    ctx->event_pool.push_back(r.a);
    ctx->event_pool.push_back(r.b);
  }
  ctx->timed.clear();
  return SHBIM_OK;
}
}  // namespace

int shbim_kernel_stats(shbim_ctx* ctx, int cls, double* ms, int64_t* launches) {
  if (!ctx) return SHBIM_ERR_ARG;
  if (cls < 0 || cls >= SHBIM_K_COUNT) return fail(ctx, SHBIM_ERR_ARG, "bad kernel class");
  if (int rc = collect_timing(ctx)) return rc;
  if (ms) *ms = ctx->class_ms[cls];
  if (launches) *launches = ctx->class_launches[cls];
  return SHBIM_OK;
}

int shbim_kernel_work(shbim_ctx* ctx, int cls, double* flops) {
  if (!ctx) return SHBIM_ERR_ARG;
  if (cls < 0 || cls >= SHBIM_K_COUNT) return fail(ctx, SHBIM_ERR_ARG, "bad kernel class");
  if (int rc = collect_timing(ctx)) return rc;
  if (flops) *flops = ctx->class_work[cls];
  return SHBIM_OK;
}

int shbim_set_field_shape(shbim_ctx* ctx, const double* G_host) {
  if (!ctx) return SHBIM_ERR_ARG;
  if (!G_host) return fail(ctx, SHBIM_ERR_ARG, "null field shape");
  double mx = 0.0;
  for (int k = 0; k < 9; ++k) {
    if (!std::isfinite(G_host[k])) return fail(ctx, SHBIM_ERR_ARG, "field shape not finite");
    mx = std::max(mx, std::fabs(G_host[k]));
  }
  const double tol = 1e-12 * mx;
  if (std::fabs(G_host[1] - G_host[3]) > tol || std::fabs(G_host[2] - G_host[6]) > tol ||
      std::fabs(G_host[5] - G_host[7]) > tol)
    return fail(ctx, SHBIM_ERR_ARG, "field shape not symmetric (the far field must be curl-free)");
  if (std::fabs(G_host[0] + G_host[4] + G_host[8]) > tol)
    return fail(ctx, SHBIM_ERR_ARG, "field shape not traceless (the far field must be divergence-free)");
  const double g[6] = {G_host[0], 0.5 * (G_host[1] + G_host[3]), 0.5 * (G_host[2] + G_host[6]), G_host[4],
                       0.5 * (G_host[5] + G_host[7]), G_host[8]};
  std::memcpy(ctx->field_g, g, sizeof(g));
  return SHBIM_OK;
}

int shbim_set_quantized_pairs(shbim_ctx* ctx, int on) {
  if (!ctx) return SHBIM_ERR_ARG;
  ctx->dq_pairs = on != 0;
  for (auto& c : ctx->pair_cfg) c.fp64class_splits = 0;  // the other kernel's occupancy
  ctx->geom_version++;  // captured operator graphs hold the other kernel
  return SHBIM_OK;
}

int shbim_set_equation_of_state(shbim_ctx* ctx, int law) {
  if (!ctx) return SHBIM_ERR_ARG;
  if (law != SHBIM_EOS_LANGMUIR && law != SHBIM_EOS_LINEAR) return fail(ctx, SHBIM_ERR_ARG, "unknown equation of state");
  ctx->eos = law;
  return SHBIM_OK;
}

int shbim_electric_rhs(shbim_ctx* ctx, const double* E_u_host, double E_q, double* out_dev, void* stream) {
  if (!ctx) return SHBIM_ERR_ARG;
  if (ctx->n_drops == 0) return fail(ctx, SHBIM_ERR_ARG, "no drops set");
  if (!E_u_host || !out_dev) return fail(ctx, SHBIM_ERR_ARG, "null pointer");
  cudaStream_t s = (cudaStream_t)stream;
  const double R = ctx->opts.R;
  FieldShape G;
  std::memcpy(G.g, ctx->field_g, sizeof(G.g));
  k_field_normal<<<(unsigned)((ctx->ntarget + 255) / 256), 256, 0, s>>>(
      ctx->geo.tgt, ctx->ntarget, E_u_host[0], E_u_host[1], E_u_host[2], E_q, G, R / (R + 1.0), ctx->grid_out);
  SHBIM_CHECK_LAUNCH(ctx, "k_field_normal");
  for (const DegreeGroup& G : ctx->groups) {
    const DropList L = G.targets();
    int rc = sht_analysis(ctx, G.tab->base, G.n, ctx->grid_out, 0, true, out_dev, ncoef(G.tab->p), s, 1, &L);
    if (rc) return rc;
  }
  return SHBIM_OK;
}

}  // extern "C"
