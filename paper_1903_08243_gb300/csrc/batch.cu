// Many operators in one call: grouped persistent launches, captured in a
// CUDA graph for replay.
//
// Forms that share (degree, quadrature, kind, precision) on hexahedra with
// the atomic scatter form a class; one persistent launch per class walks the
// batches of all its forms (hex_apply_group_kernel).  Every other form is
// applied by its own launch.  mfa_batch_create records the zeroing of all
// outputs and all launches once into a CUDA graph; mfa_batch_apply replays it
// as one graph launch on the context stream.
#include <map>
#include <tuple>
#include <vector>

#include "mfa_internal.h"

struct mfa_batch {
  mfa_ctx* ctx = nullptr;
  int device = 0;  // CUDA device of the handle's memory (destroy does not read ctx)
  struct Group {
    int n, kind, prec;
    mfa::HexTables tb;
    mfa::HexApplyArgs* d_items = nullptr;
    int64_t* d_first = nullptr;
    int nitems = 0;
    int64_t total = 0;
    int max_blocks = 0;  // smallest positive grid cap of the members (0: none)
  };
  std::vector<Group> groups;
  std::vector<int> singles;  // forms applied one by one
  std::vector<mfa_form*> forms;
  std::vector<const double*> xs;
  std::vector<double*> ys;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

int enqueue(mfa_batch* b, cudaStream_t s) {
  for (size_t k = 0; k < b->forms.size(); ++k) {
    const int64_t ndof = b->forms[k]->space->nnode * b->forms[k]->space->ncomp;
    if (cudaMemsetAsync(b->ys[k], 0, sizeof(double) * ndof, s) != cudaSuccess)
      return mfa::set_error(MFA_ERR_CUDA, "mfa_batch: zeroing an output failed");
  }
  for (auto& g : b->groups) {
    cudaError_t e = mfa::hex_group_launch(g.n, g.kind, g.prec, g.tb, g.d_items, g.d_first, g.nitems, g.total,
                                          mfa::GridBudget{b->ctx->sm_count, g.max_blocks}, s);
    if (e != cudaSuccess) return mfa::set_error(MFA_ERR_CUDA, cudaGetErrorString(e));
  }
  for (int k : b->singles) {
    int rc = mfa::apply_form(b->forms[k], b->xs[k], b->ys[k], s);
    if (rc) return rc;
  }
  return MFA_OK;
}

int build(mfa_ctx* ctx, int n, mfa_form* const* forms, const double* const* xs, double* const* ys, mfa_batch* b) {
  b->ctx = ctx;
  b->device = ctx->device;
  std::map<std::tuple<int, int, int>, std::vector<int>> classes;
  for (int k = 0; k < n; ++k) {
    mfa_form* f = forms[k];
    if (!f || !xs[k] || !ys[k]) return mfa::set_error(MFA_ERR_ARG, "mfa_batch: NULL form or vector");
    if (f->ctx != ctx) return mfa::set_error(MFA_ERR_ARG, "mfa_batch: form of another context");
    if ((const void*)xs[k] == (const void*)ys[k]) return mfa::set_error(MFA_ERR_ARG, "mfa_batch: x and y alias");
    if (f->p.kind == MFA_FORM_HYPER_JAC && !f->d_coef)
      return mfa::set_error(MFA_ERR_ARG, "mfa_batch: HYPER_JAC without coefficient");
    b->forms.push_back(f);
    b->xs.push_back(xs[k]);
    b->ys.push_back(ys[k]);
    const bool groupable = f->space->mesh->cell_type == MFA_CELL_HEX8 && f->space->ncomp == 1 && !f->d_dir_mask &&
                           f->d_geom != nullptr &&
                           f->scatter == MFA_SCATTER_ATOMIC && f->nq1 == f->space->degree + 1;
    if (groupable) classes[{f->space->degree + 1, f->p.kind, f->p.precision}].push_back(k);
    else b->singles.push_back(k);
  }
  for (auto& [key, members] : classes) {
    mfa_batch::Group g{};
    g.n = std::get<0>(key);
    g.kind = std::get<1>(key);
    g.prec = std::get<2>(key);
    g.tb = forms[members[0]]->hex;
    const int cb = g.prec != MFA_PREC_FP64          ? mfa::hex_line_cells_per_block(g.n)
                   : mfa::hex_use_eo(g.n, g.n, g.prec) ? mfa::hex_eo_cells_per_block(g.n)
                                                       : mfa::hex_cells_per_block(g.n, g.n);
    std::vector<mfa::HexApplyArgs> items;
    std::vector<int64_t> first{0};
    for (int k : members) {
      mfa_form* f = forms[k];
      if (g.prec != MFA_PREC_FP64 &&
          f->gstride > mfa::line_geom_stride_max(g.n, mfa::hex_geom_entries(g.kind), g.prec == MFA_PREC_BF16 ? 2 : 4))
        return mfa::set_error(MFA_ERR_UNSUPPORTED, "mfa_batch: factor block larger than the line kernels' stage");
      mfa::HexApplyArgs a{xs[k], ys[k], f->space->d_cell_node, f->d_geom,     nullptr,
                          f->space->mesh->ncell, ctx->d_err, f->gstride};
      items.push_back(a);
      if (f->launch.max_blocks > 0 && (g.max_blocks == 0 || f->launch.max_blocks < g.max_blocks))
        g.max_blocks = f->launch.max_blocks;
      first.push_back(first.back() + (f->space->mesh->ncell + cb - 1) / cb);
    }
    g.nitems = (int)items.size();
    g.total = first.back();
    if (cudaMalloc((void**)&g.d_items, sizeof(mfa::HexApplyArgs) * items.size()) != cudaSuccess ||
        cudaMalloc((void**)&g.d_first, sizeof(int64_t) * first.size()) != cudaSuccess) {
      b->groups.push_back(g);
      return mfa::set_error(MFA_ERR_OOM, "mfa_batch: work tables");
    }
    b->groups.push_back(g);
    if (cudaMemcpy(g.d_items, items.data(), sizeof(mfa::HexApplyArgs) * items.size(), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(g.d_first, first.data(), sizeof(int64_t) * first.size(), cudaMemcpyHostToDevice) != cudaSuccess)
      return mfa::set_error(MFA_ERR_CUDA, "mfa_batch: copying work tables");
  }
  return MFA_OK;
}

void release(mfa_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (auto& g : b->groups) {
    cudaFree(g.d_items);
    cudaFree(g.d_first);
  }
  delete b;
}

}  // namespace

extern "C" {

int mfa_apply_batched(mfa_ctx* ctx, int n, mfa_form* const* forms, const double* const* xs, double* const* ys) {
  if (!ctx || n < 0 || (n > 0 && (!forms || !xs || !ys))) return mfa::set_error(MFA_ERR_ARG, "mfa_apply_batched: bad arguments");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return mfa::set_error(MFA_ERR_CUDA, "mfa_apply_batched: cudaSetDevice");
  mfa_batch* b = new mfa_batch();
  int rc = build(ctx, n, forms, xs, ys, b);
  if (!rc) rc = enqueue(b, ctx->stream);
  if (!rc && cudaStreamSynchronize(ctx->stream) != cudaSuccess)
    rc = mfa::set_error(MFA_ERR_CUDA, "mfa_apply_batched: synchronize");
  release(b);
  return rc;
}

int mfa_batch_create(mfa_ctx* ctx, int n, mfa_form* const* forms, const double* const* xs, double* const* ys,
                     mfa_batch** out) {
  if (!ctx || !out || n < 0 || (n > 0 && (!forms || !xs || !ys)))
    return mfa::set_error(MFA_ERR_ARG, "mfa_batch_create: bad arguments");
  *out = nullptr;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return mfa::set_error(MFA_ERR_CUDA, "mfa_batch_create: cudaSetDevice");
  mfa_batch* b = new mfa_batch();
  int rc = build(ctx, n, forms, xs, ys, b);
  // one eager pass initialises every kernel's launch attributes outside the capture
  if (!rc) rc = enqueue(b, ctx->stream);
  if (!rc && cudaStreamSynchronize(ctx->stream) != cudaSuccess) rc = mfa::set_error(MFA_ERR_CUDA, "synchronize");
  cudaStream_t cs = nullptr;
  if (!rc && cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess)
    rc = mfa::set_error(MFA_ERR_CUDA, "mfa_batch_create: capture stream");
  if (!rc && cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    rc = mfa::set_error(MFA_ERR_CUDA, "mfa_batch_create: begin capture");
  if (!rc) {
    int rc2 = enqueue(b, cs);
    cudaError_t e = cudaStreamEndCapture(cs, &b->graph);
    rc = rc2 ? rc2 : (e == cudaSuccess ? MFA_OK : mfa::set_error(MFA_ERR_CUDA, "mfa_batch_create: end capture"));
  }
  if (!rc && cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess)
    rc = mfa::set_error(MFA_ERR_CUDA, "mfa_batch_create: instantiate graph");
  if (cs) cudaStreamDestroy(cs);
  if (rc) {
    release(b);
    return rc;
  }
  *out = b;
  return MFA_OK;
}

int mfa_batch_apply(mfa_ctx* ctx, mfa_batch* b) {
  if (!ctx || !b || b->ctx != ctx) return mfa::set_error(MFA_ERR_ARG, "mfa_batch_apply: bad arguments");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return mfa::set_error(MFA_ERR_CUDA, "mfa_batch_apply: cudaSetDevice");
  cudaError_t e = cudaGraphLaunch(b->exec, ctx->stream);
  return e == cudaSuccess ? MFA_OK : mfa::set_error(MFA_ERR_CUDA, cudaGetErrorString(e));
}

int mfa_batch_info(const mfa_batch* b, int* nlaunch_groups, int* nsingles) {
  if (!b) return mfa::set_error(MFA_ERR_ARG, "mfa_batch_info: NULL batch");
  if (nlaunch_groups) *nlaunch_groups = (int)b->groups.size();
  if (nsingles) *nsingles = (int)b->singles.size();
  return MFA_OK;
}

int mfa_batch_destroy(mfa_batch* b) {
  if (!b) return MFA_OK;
  cudaSetDevice(b->device);
  release(b);
  return MFA_OK;
}

}  // extern "C"
