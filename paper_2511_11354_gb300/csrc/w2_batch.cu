// Batching form: many independent problems of uneven grid sizes and
// interaction strengths advanced together.  Each instance is an ordinary
// FP32 precision-form context (its own arrays and tables); one step of the
// whole batch is a fixed sequence of persistent kernels, each striding over
// the flattened (instance, work item) list of every instance (or of every
// instance of one momentum size, for the kernels specialised on it), captured
// once into a CUDA graph.  Grid sizes are chosen by timing candidates on the
// real batch (w2_batch_autotune).
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "w2_internal.cuh"

using namespace w2;

namespace {

struct Class {  // instances sharing one momentum size
  int nk = 0;
  std::vector<int> inst;
  int *d_inst = nullptr, *d_off_x = nullptr, *d_off_slab = nullptr;
  int items_x = 0, items_slab = 0;
  int grid_theta = 0, grid_adv0 = 0, grid_adv1 = 0;
  int nxmax = 0, nxmin = 1 << 30;
};

}  // namespace

struct w2_batch {
  int n = 0;
  std::vector<w2_ctx *> inst;
  cudaStream_t stream = nullptr, cap = nullptr;
  TabArgs *d_tab = nullptr;
  BXsum *d_xs_f = nullptr, *d_xs_ft = nullptr;
  Theta32Args *d_th = nullptr;
  Adv32Args *d_adv = nullptr;
  int *d_off_x = nullptr, *d_off_tab = nullptr;
  int items_x = 0, items_tab = 0;
  int grid_xsum = 0, grid_tab = 0;
  int nxmax = 0, mmax = 0, sms = 0;
  std::vector<Class> cls;
  cudaGraphExec_t graph = nullptr;
  bool graph_ready = false;
  bool tab_dirty = true;  // table arguments carry the potentials' weights
  w2_status sticky = W2_OK;
};

#define WB_TRY(call)                  \
  do {                                \
    if ((call) != cudaSuccess) {      \
      b->sticky = W2_ERR_CUDA;        \
      return W2_ERR_CUDA;             \
    }                                 \
  } while (0)

static void batch_free(w2_batch *b) {
  if (b->graph_ready) cudaGraphExecDestroy(b->graph);
  void *ptrs[] = {b->d_tab, b->d_xs_f, b->d_xs_ft, b->d_th, b->d_adv, b->d_off_x, b->d_off_tab};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  for (auto &c : b->cls) {
    if (c.d_inst) cudaFree(c.d_inst);
    if (c.d_off_x) cudaFree(c.d_off_x);
    if (c.d_off_slab) cudaFree(c.d_off_slab);
  }
  for (w2_ctx *c : b->inst)
    if (c) w2_destroy(c);
  if (b->cap) cudaStreamDestroy(b->cap);
}

template <typename T>
static cudaError_t upload(T **dst, const std::vector<T> &v) {
  cudaError_t e = cudaMalloc((void **)dst, sizeof(T) * std::max<size_t>(v.size(), 1));
  if (e == cudaSuccess) e = cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
  return e;
}

extern "C" void w2_batch_destroy(w2_batch *b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  batch_free(b);
  delete b;
}

extern "C" w2_status w2_batch_create(const w2_config *cfgs, int32_t n, void *cuda_stream, w2_batch **out) {
  if (!out) return W2_ERR_ARG;
  *out = nullptr;
  if (!cfgs || n <= 0 || n > 4096) return W2_ERR_ARG;
  for (int i = 0; i < n; ++i)
    if (cfgs[i].precision != W2_F32_TF32X3) return W2_ERR_UNSUPPORTED;
  w2_batch *b = new (std::nothrow) w2_batch();
  if (!b) return W2_ERR_OOM;
  b->n = n;
  b->stream = (cudaStream_t)cuda_stream;
  b->inst.assign(n, nullptr);
  for (int i = 0; i < n; ++i) {
    w2_status st = w2_create(&cfgs[i], cuda_stream, &b->inst[i]);
    if (st != W2_OK) {
      batch_free(b);
      delete b;
      return st;
    }
  }
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) {
    batch_free(b);
    delete b;
    return W2_ERR_CUDA;
  }
  b->sms = prop.multiProcessorCount;

  std::vector<TabArgs> tab(n);
  std::vector<BXsum> xf(n), xft(n);
  std::vector<Theta32Args> th(2 * n);
  std::vector<Adv32Args> adv(2 * n);
  std::vector<int> off_x(n + 1, 0), off_tab(n + 1, 0);
  for (int i = 0; i < n; ++i) {
    w2_ctx *c = b->inst[i];
    const int W = 2 * c->nk - 1;
    float *f = (float *)c->f, *g = (float *)c->g, *t1 = (float *)c->t1, *t2 = (float *)c->t2;
    tab[i] = tab_args(c, c->xsum, 0);
    xf[i] = BXsum{f, c->xsum, c->nk};
    xft[i] = BXsum{g, c->xsum, c->nk};
    Theta32Args &p = th[2 * i], &q = th[2 * i + 1];
    p.nx = c->nx;
    p.in = f;
    p.base = nullptr;
    p.h = nullptr;
    p.out = g;
    p.K1 = c->K;
    p.K2 = c->K + (size_t)c->nx * W;
    p.K12 = c->K12;
    p.half_tau = (float)(0.5 * c->tau);
    q = p;
    q.in = g;
    q.base = f;
    q.h = t1;
    q.out = f;
    Adv32Args a0 = adv32_args(c), a1 = adv32_args(c);
    a0.f = f;
    a0.g = g;
    a0.d2 = t1;
    a0.g2 = t2;
    a1.f = f;
    a1.d2in = t1;
    a1.g2in = t2;
    a1.ft = g;
    a1.dh = t1;
    adv[2 * i] = a0;
    adv[2 * i + 1] = a1;
    off_x[i + 1] = off_x[i] + c->nx * c->nx;
    off_tab[i + 1] = off_tab[i] + 2 * c->nx;
    b->nxmax = std::max(b->nxmax, c->nx);
    b->mmax = std::max(b->mmax, c->M);
    // momentum-size classes
    int k = -1;
    for (size_t q2 = 0; q2 < b->cls.size(); ++q2)
      if (b->cls[q2].nk == c->nk) k = (int)q2;
    if (k < 0) {
      b->cls.emplace_back();
      k = (int)b->cls.size() - 1;
      b->cls[k].nk = c->nk;
    }
    b->cls[k].inst.push_back(i);
    b->cls[k].nxmax = std::max(b->cls[k].nxmax, c->nx);
    b->cls[k].nxmin = std::min(b->cls[k].nxmin, c->nx);
  }
  b->items_x = off_x[n];
  b->items_tab = off_tab[n];
  cudaError_t e = upload(&b->d_tab, tab);
  if (e == cudaSuccess) e = upload(&b->d_xs_f, xf);
  if (e == cudaSuccess) e = upload(&b->d_xs_ft, xft);
  if (e == cudaSuccess) e = upload(&b->d_th, th);
  if (e == cudaSuccess) e = upload(&b->d_adv, adv);
  if (e == cudaSuccess) e = upload(&b->d_off_x, off_x);
  if (e == cudaSuccess) e = upload(&b->d_off_tab, off_tab);
  for (auto &c : b->cls) {
    std::vector<int> ox(c.inst.size() + 1, 0), os(c.inst.size() + 1, 0);
    for (size_t q = 0; q < c.inst.size(); ++q) {
      w2_ctx *ci = b->inst[c.inst[q]];
      ox[q + 1] = ox[q] + ci->nx * ci->nx;
      os[q + 1] = os[q] + ci->nk * ci->nx * adv_items_per_line_f32(ci->nk);
    }
    c.items_x = ox.back();
    c.items_slab = os.back();
    if (e == cudaSuccess) e = upload(&c.d_inst, c.inst);
    if (e == cudaSuccess) e = upload(&c.d_off_x, ox);
    if (e == cudaSuccess) e = upload(&c.d_off_slab, os);
    // default grids: two waves of CTAs over the SMs, at most one per item
    c.grid_theta = std::min(c.items_x, 2 * b->sms);
    c.grid_adv0 = std::min(c.items_slab, 4 * b->sms);
    c.grid_adv1 = std::min(c.items_slab, 4 * b->sms);
  }
  b->grid_xsum = std::min(b->items_x, 8 * b->sms);
  b->grid_tab = std::min(b->items_tab, 4 * b->sms);
  if (e != cudaSuccess) {
    batch_free(b);
    delete b;
    return e == cudaErrorMemoryAllocation ? W2_ERR_OOM : W2_ERR_CUDA;
  }
  *out = b;
  return W2_OK;
}

static bool index_ok(const w2_batch *b, int i) { return b && i >= 0 && i < b->n; }

extern "C" w2_status w2_batch_set_potentials(w2_batch *b, int32_t i, w2_fn vext, void *ue, w2_fn vee, void *ui,
                                             double gamma, double c_hartree, double c_xc) {
  if (!index_ok(b, i)) return W2_ERR_ARG;
  if (b->sticky) return b->sticky;
  b->tab_dirty = true;
  return w2_set_potentials(b->inst[i], vext, ue, vee, ui, gamma, c_hartree, c_xc);
}

extern "C" w2_status w2_batch_set_state(w2_batch *b, int32_t i, const void *f, int32_t on_device) {
  if (!index_ok(b, i)) return W2_ERR_ARG;
  if (b->sticky) return b->sticky;
  return w2_set_state(b->inst[i], f, on_device);
}

extern "C" w2_status w2_batch_get_state(w2_batch *b, int32_t i, void *f, int32_t on_device) {
  if (!index_ok(b, i)) return W2_ERR_ARG;
  if (b->sticky) return b->sticky;
  return w2_get_state(b->inst[i], f, on_device);
}

extern "C" w2_status w2_batch_observables(w2_batch *b, int32_t i, w2_obs *out, double *n1, double *n12) {
  if (!index_ok(b, i)) return W2_ERR_ARG;
  if (b->sticky) return b->sticky;
  return w2_observables(b->inst[i], out, n1, n12);
}

// Kernels of one batch step, in order:
//   per-X sums (all) ; tables (all) ; Theta predictor (per class) ;
//   shift x2 (per class) ; shift x1 + combination (per class) ;
//   per-X sums of f~ (all) ; tables (all) ; Theta corrector (per class)
static cudaError_t enqueue_batch_step(w2_batch *b, cudaStream_t s) {
  cudaError_t e;
  if ((e = launch_bxsum(b->d_xs_f, b->d_off_x, b->n, b->grid_xsum, s)) != cudaSuccess) return e;
  if ((e = launch_btables(b->d_tab, b->d_off_tab, b->n, b->grid_tab, b->nxmax, b->mmax, s)) != cudaSuccess) return e;
  for (auto &c : b->cls) {
    BatchLaunch bl{c.grid_theta, c.d_inst, c.d_off_x, (int)c.inst.size()};
    if ((e = launch_btheta_f32(c.nk, 0, bl, b->d_th, s)) != cudaSuccess) return e;
  }
  for (auto &c : b->cls) {
    BatchLaunch bl{c.grid_adv0, c.d_inst, c.d_off_slab, (int)c.inst.size()};
    if ((e = launch_badv_f32(c.nk, 0, bl, b->d_adv, c.nxmax, adv32_pieces(c.nxmax), s)) != cudaSuccess) return e;
  }
  for (auto &c : b->cls) {
    BatchLaunch bl{c.grid_adv1, c.d_inst, c.d_off_slab, (int)c.inst.size()};
    if ((e = launch_badv_f32(c.nk, 1, bl, b->d_adv, c.nxmax, adv32_pieces(c.nxmax), s)) != cudaSuccess) return e;
  }
  if ((e = launch_bxsum(b->d_xs_ft, b->d_off_x, b->n, b->grid_xsum, s)) != cudaSuccess) return e;
  if ((e = launch_btables(b->d_tab, b->d_off_tab, b->n, b->grid_tab, b->nxmax, b->mmax, s)) != cudaSuccess) return e;
  for (auto &c : b->cls) {
    BatchLaunch bl{c.grid_theta, c.d_inst, c.d_off_x, (int)c.inst.size()};
    if ((e = launch_btheta_f32(c.nk, 1, bl, b->d_th, s)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

static w2_status ready(w2_batch *b) {
  if (b->sticky) return b->sticky;
  for (w2_ctx *c : b->inst)
    if (!c->have_pot || !c->have_state) return W2_ERR_STATE;
  if (b->tab_dirty) {
    // the kernels read their arguments from device memory at run time, so a
    // captured step sees the refreshed weights without being captured again
    std::vector<TabArgs> tab(b->n);
    for (int i = 0; i < b->n; ++i) tab[i] = tab_args(b->inst[i], b->inst[i]->xsum, 0);
    if (cudaMemcpyAsync(b->d_tab, tab.data(), sizeof(TabArgs) * b->n, cudaMemcpyHostToDevice, b->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess) {
      b->sticky = W2_ERR_CUDA;
      return W2_ERR_CUDA;
    }
    b->tab_dirty = false;
  }
  return W2_OK;
}

extern "C" w2_status w2_batch_step(w2_batch *b, int32_t nsteps) {
  if (!b || nsteps < 0) return W2_ERR_ARG;
  w2_status st = ready(b);
  if (st) return st;
  if (nsteps == 0) return W2_OK;
  if (!b->graph_ready) {
    cudaGraph_t graph;
    WB_TRY(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = enqueue_batch_step(b, b->cap);
    cudaError_t e2 = cudaStreamEndCapture(b->cap, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (e2 == cudaSuccess) cudaGraphDestroy(graph);
      b->sticky = W2_ERR_CUDA;
      return W2_ERR_CUDA;
    }
    e = cudaGraphInstantiate(&b->graph, graph, 0);
    cudaGraphDestroy(graph);
    WB_TRY(e);
    b->graph_ready = true;
  }
  for (int s = 0; s < nsteps; ++s) WB_TRY(cudaGraphLaunch(b->graph, b->stream));
  for (w2_ctx *c : b->inst) c->steps += nsteps;
  return W2_OK;
}

// Time one launch configuration: the best of `reps` launches, in ms.
template <typename F>
static float time_best(cudaStream_t s, F launch, int reps, cudaError_t *err) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int r = 0; r < reps + 1; ++r) {
    cudaEventRecord(e0, s);
    cudaError_t e = launch();
    cudaEventRecord(e1, s);
    if (e != cudaSuccess) *err = e;
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (r > 0) best = std::min(best, ms);  // the first launch warms up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}

extern "C" w2_status w2_batch_autotune(w2_batch *b, int32_t *grids_out, int32_t grids_len) {
  if (!b) return W2_ERR_ARG;
  w2_status st = ready(b);
  if (st) return st;
  cudaStream_t s = b->stream;
  cudaError_t err = cudaSuccess;
  const int mult[] = {1, 2, 3, 4, 6, 8, 12, 16};
  auto candidates = [&](int items) {
    std::vector<int> v;
    for (int m : mult) {
      const int g = std::min(items, m * b->sms);
      if (std::find(v.begin(), v.end(), g) == v.end()) v.push_back(g);
    }
    return v;
  };
  // Each tuned kernel is free of side effects on the state: the predictor
  // sweep and the x2 pass write scratch arrays only, and the x1 pass is timed
  // writing into scratch as well (its inputs are rebuilt by the next step).
  {
    float best = 1e30f;
    int pick = b->grid_xsum;
    for (int g : candidates(b->items_x)) {
      float t = time_best(s, [&] { return launch_bxsum(b->d_xs_f, b->d_off_x, b->n, g, s); }, 2, &err);
      if (t < best) best = t, pick = g;
    }
    b->grid_xsum = pick;
  }
  {
    float best = 1e30f;
    int pick = b->grid_tab;
    for (int g : candidates(b->items_tab)) {
      float t = time_best(
          s, [&] { return launch_btables(b->d_tab, b->d_off_tab, b->n, g, b->nxmax, b->mmax, s); }, 2, &err);
      if (t < best) best = t, pick = g;
    }
    b->grid_tab = pick;
  }
  for (auto &c : b->cls) {
    const int m = (int)c.inst.size();
    float best = 1e30f;
    int pick = c.grid_theta;
    for (int g : candidates(c.items_x)) {
      BatchLaunch bl{g, c.d_inst, c.d_off_x, m};
      float t = time_best(s, [&] { return launch_btheta_f32(c.nk, 0, bl, b->d_th, s); }, 2, &err);
      if (t < best) best = t, pick = g;
    }
    c.grid_theta = pick;
    best = 1e30f;
    pick = c.grid_adv0;
    for (int g : candidates(c.items_slab)) {
      BatchLaunch bl{g, c.d_inst, c.d_off_slab, m};
      float t = time_best(s, [&] { return launch_badv_f32(c.nk, 0, bl, b->d_adv, c.nxmax, adv32_pieces(c.nxmax), s); }, 2, &err);
      if (t < best) best = t, pick = g;
    }
    c.grid_adv0 = pick;
    // the x1 pass has the same item structure and a larger working set; tune it
    // separately after restoring its inputs with one x2 pass
    best = 1e30f;
    pick = c.grid_adv1;
    for (int g : candidates(c.items_slab)) {
      BatchLaunch b0{c.grid_adv0, c.d_inst, c.d_off_slab, m};
      BatchLaunch bl{g, c.d_inst, c.d_off_slab, m};
      float t = time_best(
          s,
          [&] {
            cudaError_t e0 = launch_badv_f32(c.nk, 0, b0, b->d_adv, c.nxmax, adv32_pieces(c.nxmax), s);
            return e0 != cudaSuccess ? e0 : launch_badv_f32(c.nk, 1, bl, b->d_adv, c.nxmax, adv32_pieces(c.nxmax), s);
          },
          2, &err);
      if (t < best) best = t, pick = g;
    }
    c.grid_adv1 = pick;
  }
  if (err != cudaSuccess) {
    b->sticky = W2_ERR_CUDA;
    return W2_ERR_CUDA;
  }
  if (b->graph_ready) {  // the captured step used the old grids
    cudaGraphExecDestroy(b->graph);
    b->graph_ready = false;
  }
  if (grids_out && grids_len > 0) {
    std::vector<int> v = {b->grid_xsum, b->grid_tab};
    for (auto &c : b->cls) {
      v.push_back(c.nk);
      v.push_back(c.grid_theta);
      v.push_back(c.grid_adv0);
      v.push_back(c.grid_adv1);
    }
    for (int q = 0; q < grids_len; ++q) grids_out[q] = q < (int)v.size() ? v[q] : 0;
  }
  return W2_OK;
}
