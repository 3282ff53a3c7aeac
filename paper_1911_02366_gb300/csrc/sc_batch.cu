// Batched condensation of elements of uneven polynomial order: the condensation set-up of
// several assembled systems (each of one order N, mixed arm) run together, not in the
// paper (which condenses one element after another, Sec. 3.2).
//
// Every element of every system becomes one item (its sizes and block addresses).  The
// Gauss-Jordan inverses, the S_ee copies, the LU panel steps, the pivot permutations, the
// diagonal-block inverses and the solve layout run as grouped launches over all items
// (one CTA per item).  Items are ordered by decreasing block size, so that the orders
// N >= 5 (n_i > 136, n_b > 496) form a prefix that takes the large-block kernels (blocked
// Gauss-Jordan, shared-memory LU panels) while the rest run register-resident.  The TF32 tensor-core
// products (Y^T, S_ee, the LU trailing updates) run per order through tables of block
// addresses, with the N-tile width of each chosen by timing the candidates on the
// batch's own data (autotune).  The whole sequence can be captured once into a CUDA
// graph, on a stream the batch owns, and replayed for every new set of systems.
#include <algorithm>
#include <map>
#include <string>
#include <tuple>

#include "sc_internal.cuh"

namespace {

constexpr int kBnChoices[3] = {64, 144, 256};

struct OrderClass {
  int ni = 0, nb = 0, lda = 0, ldi = 0, lds = 0, count = 0;
  int bn_y = 256, bn_s = 256, bn_t = 256;  // N-tile widths of the three products
  size_t off_y = 0, off_s = 0;             // offsets of the address tables (3 x count each)
  std::vector<size_t> off_t;               // per LU step with a trailing update
};

}  // namespace

struct sc_batch {
  std::vector<sc_ctx*> ctx;
  cudaStream_t stream = nullptr;   // the systems' stream
  cudaStream_t cap = nullptr;      // the batch's own stream (graph capture and replay)
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  std::vector<CondItem> items;
  std::vector<OrderClass> cls;
  CondItem* d_items = nullptr;
  void** d_ptrs = nullptr;
  std::vector<void*> h_ptrs;
  int max_ni = 0, max_nb = 0;
  int nbig_gj = 0, nbig_lu = 0;  // leading items that take the large-block GJ / LU panel kernels
  int* d_status = nullptr;
  bool tuned = false;
  long long grouped_launches = 0;  // kernel launches of one run outside the systems' own
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

cudaError_t run_products_y(sc_batch* b, cudaStream_t st, const OrderClass& oc, int bn) {
  const float* const* A = reinterpret_cast<const float* const*>(b->d_ptrs + oc.off_y);
  return sc::gemm_tf32_ptrs(st, oc.nb, oc.ni, oc.ni, 1.0f, A, oc.lda, true, A + oc.count, oc.ldi, true, 0.0f,
                            reinterpret_cast<float* const*>(b->d_ptrs + oc.off_y + 2 * oc.count), oc.ldi, oc.count,
                            bn, b->d_status);
}

cudaError_t run_products_s(sc_batch* b, cudaStream_t st, const OrderClass& oc, int bn) {
  const float* const* A = reinterpret_cast<const float* const*>(b->d_ptrs + oc.off_s);
  return sc::gemm_tf32_ptrs(st, oc.nb, oc.nb, oc.ni, -1.0f, A, oc.lda, false, A + oc.count, oc.ldi, true, 1.0f,
                            reinterpret_cast<float* const*>(b->d_ptrs + oc.off_s + 2 * oc.count), oc.lds, oc.count,
                            bn, b->d_status);
}

cudaError_t run_trailing(sc_batch* b, cudaStream_t st, const OrderClass& oc, int step, int bn) {
  const int k0 = 32 * step, rest = oc.nb - k0 - 32;
  const size_t o = oc.off_t[step];
  const float* const* A = reinterpret_cast<const float* const*>(b->d_ptrs + o);
  return sc::gemm_tf32_ptrs(st, rest, rest, 32, -1.0f, A, oc.lds, false, A + oc.count, oc.lds, false, 1.0f,
                            reinterpret_cast<float* const*>(b->d_ptrs + o + 2 * oc.count), oc.lds, oc.count, bn,
                            b->d_status);
}

// The whole set-up on stream st, in the order of sc_condense.
cudaError_t run_all(sc_batch* b, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  for (sc_ctx* c : b->ctx) {
    const Geo& G = c->G;
    const cudaStream_t own = c->stream;
    c->stream = st;  // the per-system conversions go to the same stream as the rest
    if (e == cudaSuccess) e = sc::pack_own(c);  // also writes the FP32 own blocks
    if (e == cudaSuccess) e = sc::to_float(c, c->X, c->X32, (size_t)G.K * G.NP * 25);
    c->stream = own;
  }
  const int n = (int)b->items.size();
  // grouped launches of this run: GJ, copy, 3 finishing kernels, the products and the panels
  long long nl = sc::grouped_gj_launches(b->nbig_gj, n, b->max_ni) + 4 + 2 * (long long)b->cls.size();
  for (int step = 0; 32 * step < b->max_nb; ++step) {
    nl += (b->nbig_lu > 0 ? 1 : 0) + (n > b->nbig_lu ? 1 : 0);
    for (const OrderClass& oc : b->cls) nl += step < (int)oc.off_t.size() ? 1 : 0;
  }
  b->grouped_launches = nl;
  if (e == cudaSuccess) e = sc::grouped_gj(st, b->d_items, n, b->nbig_gj, b->max_ni);
  for (const OrderClass& oc : b->cls)
    if (e == cudaSuccess) e = run_products_y(b, st, oc, oc.bn_y);
  if (e == cudaSuccess) e = sc::grouped_copy_bb(st, b->d_items, n);
  for (const OrderClass& oc : b->cls)
    if (e == cudaSuccess) e = run_products_s(b, st, oc, oc.bn_s);
  for (int step = 0; 32 * step < b->max_nb && e == cudaSuccess; ++step) {
    e = sc::grouped_lu_panel(st, b->d_items, n, b->nbig_lu, 32 * step, b->max_nb);
    for (const OrderClass& oc : b->cls)
      if (e == cudaSuccess && step < (int)oc.off_t.size()) e = run_trailing(b, st, oc, step, oc.bn_t);
  }
  if (e == cudaSuccess) e = sc::grouped_finish(st, b->d_items, n, b->max_nb);
  return e;
}

// Time one product for each candidate width on the batch's data; keep the fastest.
template <class F>
int pick_width(cudaStream_t st, F&& launch) {
  cudaEvent_t t0, t1;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  int best = 256;
  float best_ms = 1e30f;
  for (int bn : kBnChoices) {
    if (launch(bn) != cudaSuccess) continue;  // warm-up
    cudaEventRecord(t0, st);
    for (int r = 0; r < 2; ++r) launch(bn);
    cudaEventRecord(t1, st);
    cudaEventSynchronize(t1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t0, t1);
    if (ms < best_ms) { best_ms = ms; best = bn; }
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  return best;
}

sc_status batch_fail(sc_batch* b, sc_status s, const std::string& msg) {
  if (!b->ctx.empty()) b->ctx[0]->err = "batched condensation: " + msg;
  return s;
}

}  // namespace

extern "C" {

sc_status sc_batch_create(sc_ctx* const* ctxs, int nctx, sc_batch** out) {
  if (!ctxs || nctx < 1 || !out) return SC_ERR_ARG;
  sc_batch* b = new sc_batch();
  b->stream = ctxs[0] ? ctxs[0]->stream : nullptr;
  for (int i = 0; i < nctx; ++i) {
    sc_ctx* c = ctxs[i];
    if (!c || !c->has_mesh || c->cfg.precision != SC_PREC_MIXED || c->cfg.precond != SC_PC_BLOCK_JACOBI ||
        c->cfg.explicit_schur || !c->cfg.tensor_cores || c->cfg.factor_fp16 || c->cfg.interior_fp64 ||
        c->stream != b->stream) {
      delete b;
      return SC_ERR_ARG;
    }
    b->ctx.push_back(c);
  }
  std::map<std::tuple<int, int, int, int, int>, int> cls_of;
  for (sc_ctx* c : b->ctx) {
    const Geo& G = c->G;
    const auto key = std::make_tuple(G.ni, G.nb, G.lda, G.ldi, G.lds);
    if (!cls_of.count(key)) {
      OrderClass oc;
      oc.ni = G.ni; oc.nb = G.nb; oc.lda = G.lda; oc.ldi = G.ldi; oc.lds = G.lds;
      cls_of[key] = (int)b->cls.size();
      b->cls.push_back(oc);
    }
    b->cls[cls_of[key]].count += G.K;
    b->max_ni = std::max(b->max_ni, G.ni);
    b->max_nb = std::max(b->max_nb, G.nb);
  }
  // items, largest blocks first so that the grouped launches start with the long CTAs
  std::vector<sc_ctx*> order = b->ctx;
  std::stable_sort(order.begin(), order.end(), [](const sc_ctx* x, const sc_ctx* y) { return x->G.nb > y->G.nb; });
  for (sc_ctx* c : order) {
    const Geo& G = c->G;
    const long long ls = sc::solve_layout_stride(G);
    for (int e = 0; e < G.K; ++e) {
      CondItem it;
      it.ni = G.ni; it.nb = G.nb; it.lda = G.lda; it.ldi = G.ldi; it.lds = G.lds; it.e = e; it.cb0 = G.cb0;
      it.Aown = c->Aown32 + (size_t)e * own_stride(G);
      it.Ainv = c->Ainv32 + (size_t)e * G.ni * G.ldi;
      it.Yt = c->Y32 + (size_t)e * G.nb * G.ldi;
      it.See = c->See32 + (size_t)e * G.nb * G.lds;
      it.Sls = c->Sls32 + (size_t)e * ls;
      it.piv = c->piv + (size_t)e * G.nb;
      it.rowperm = c->rowperm + (size_t)e * G.nb;
      it.status = nullptr;  // set once the status word exists
      it.dsc = reinterpret_cast<float*>(c->gj_scale) + (size_t)e * G.ni;
      b->items.push_back(it);
    }
  }
  // the large-block kernels take a prefix of the items (sorted by decreasing n_b, and n_i
  // grows with n_b)
  for (const CondItem& it : b->items) {
    if (sc::gj_blocked_item(it.ni)) ++b->nbig_gj;
    if (sc::lu_panel_smem_item(it.nb)) ++b->nbig_lu;
  }
  for (int i = 0; i < (int)b->items.size(); ++i)
    if (sc::gj_blocked_item(b->items[i].ni) != (i < b->nbig_gj) ||
        sc::lu_panel_smem_item(b->items[i].nb) != (i < b->nbig_lu)) {
      delete b;
      return SC_ERR_ARG;
    }
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&b->d_status), sizeof(int));
  for (CondItem& it : b->items) it.status = b->d_status;
  // address tables of the products, per order class
  for (OrderClass& oc : b->cls) {
    std::vector<const CondItem*> mine;
    for (const CondItem& it : b->items)
      if (it.ni == oc.ni && it.nb == oc.nb && it.lda == oc.lda && it.ldi == oc.ldi && it.lds == oc.lds)
        mine.push_back(&it);
    auto push3 = [&](auto fa, auto fb, auto fc) {
      const size_t off = b->h_ptrs.size();
      for (const CondItem* it : mine) b->h_ptrs.push_back((void*)fa(*it));
      for (const CondItem* it : mine) b->h_ptrs.push_back((void*)fb(*it));
      for (const CondItem* it : mine) b->h_ptrs.push_back((void*)fc(*it));
      return off;
    };
    // Y^T = A_ib^T A_ii^-T
    oc.off_y = push3([](const CondItem& it) { return it.Aown + it.cb0; }, [](const CondItem& it) { return it.Ainv; },
                     [](const CondItem& it) { return it.Yt; });
    // S_ee -= A_bi Y
    oc.off_s = push3([](const CondItem& it) { return it.Aown + (size_t)it.ni * it.lda; },
                     [](const CondItem& it) { return it.Yt; }, [](const CondItem& it) { return it.See; });
    for (int k0 = 0; oc.nb - k0 - 32 > 0; k0 += 32)
      oc.off_t.push_back(push3([k0](const CondItem& it) { return it.See + (size_t)(k0 + 32) * it.lds + k0; },
                               [k0](const CondItem& it) { return it.See + (size_t)k0 * it.lds + k0 + 32; },
                               [k0](const CondItem& it) { return it.See + (size_t)(k0 + 32) * it.lds + k0 + 32; }));
  }
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&b->d_items), b->items.size() * sizeof(CondItem));
  if (e == cudaSuccess)
    e = cudaMalloc(reinterpret_cast<void**>(&b->d_ptrs), std::max<size_t>(1, b->h_ptrs.size()) * sizeof(void*));
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_items, b->items.data(), b->items.size() * sizeof(CondItem), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_ptrs, b->h_ptrs.data(), b->h_ptrs.size() * sizeof(void*), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    sc_batch_destroy(b);
    return SC_ERR_OOM;
  }
  *out = b;
  return SC_OK;
}

sc_status sc_batch_condense(sc_batch* b, int flags) {
  if (!b) return SC_ERR_ARG;
  for (sc_ctx* c : b->ctx)
    if (!c->assembled) return batch_fail(b, SC_ERR_STATE, "a system is not assembled");
  const bool use_graph = flags & SC_BATCH_GRAPH, tune = flags & SC_BATCH_AUTOTUNE;
  const cudaStream_t st = b->stream;
  const int minus1 = -1;
  cudaError_t e = cudaMemcpyAsync(b->d_status, &minus1, sizeof(int), cudaMemcpyHostToDevice, st);
  for (sc_ctx* c : b->ctx)
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_status, &minus1, sizeof(int), cudaMemcpyHostToDevice, st);
  // all further work runs on the batch's stream, ordered after the caller's stream
  if (e == cudaSuccess) e = cudaEventRecord(b->ev_in, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(b->cap, b->ev_in, 0);
  if (e == cudaSuccess && tune && !b->tuned) {
    // the candidates run on the batch's data; the set-up below recomputes everything
    for (OrderClass& oc : b->cls) {
      oc.bn_y = pick_width(b->cap, [&](int bn) { return run_products_y(b, b->cap, oc, bn); });
      oc.bn_s = pick_width(b->cap, [&](int bn) { return run_products_s(b, b->cap, oc, bn); });
      if (!oc.off_t.empty()) oc.bn_t = pick_width(b->cap, [&](int bn) { return run_trailing(b, b->cap, oc, 0, bn); });
    }
    b->tuned = true;
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
  }
  if (e == cudaSuccess && use_graph) {
    if (!b->exec) {
      e = run_all(b, b->cap);  // also sets the kernels' shared-memory limits outside the capture
      if (e == cudaSuccess) e = cudaStreamSynchronize(b->cap);
      if (e == cudaSuccess) e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        const cudaError_t ec = run_all(b, b->cap);
        e = cudaStreamEndCapture(b->cap, &b->graph);
        if (ec != cudaSuccess) e = ec;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    }
    if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, b->cap);
  } else if (e == cudaSuccess) {
    e = run_all(b, b->cap);
  }
  if (e == cudaSuccess) e = cudaEventRecord(b->ev_out, b->cap);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, b->ev_out, 0);
  int bad = -1;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, b->d_status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return batch_fail(b, SC_ERR_CUDA, cudaGetErrorString(e));
  if (bad >= SC_TC_TIMEOUT) return batch_fail(b, SC_ERR_CUDA, "tensor-core wait timed out");
  if (bad >= 0) return batch_fail(b, SC_ERR_SINGULAR_BLOCK, "singular element block");
  for (sc_ctx* c : b->ctx) {  // the packing check of each system
    int cb = -1;
    if (cudaMemcpy(&cb, c->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
      return batch_fail(b, SC_ERR_CUDA, "status read");
    if (cb >= 0) return batch_fail(b, SC_ERR_STATE, "own-block entry outside the packed node pattern");
  }
  b->ctx[0]->launches += b->grouped_launches;  // the systems count their own conversions
  if (use_graph)
    for (sc_ctx* c : b->ctx) c->launches += 2;  // replayed packing and conversion of each system
  for (sc_ctx* c : b->ctx) {
    c->packed = true;
    c->condensed = true;
    c->ls16_ok = false;
    c->Sdiag_valid = false;
  }
  return SC_OK;
}

sc_status sc_batch_tiles(const sc_batch* b, int order_class, int* ni, int* bn_y, int* bn_s, int* bn_t) {
  if (!b || order_class < 0 || order_class >= (int)b->cls.size()) return SC_ERR_ARG;
  const OrderClass& oc = b->cls[order_class];
  if (ni) *ni = oc.ni;
  if (bn_y) *bn_y = oc.bn_y;
  if (bn_s) *bn_s = oc.bn_s;
  if (bn_t) *bn_t = oc.bn_t;
  return SC_OK;
}

void sc_batch_destroy(sc_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  cudaFree(b->d_items);
  cudaFree(b->d_ptrs);
  cudaFree(b->d_status);
  delete b;
}

}  // extern "C"
