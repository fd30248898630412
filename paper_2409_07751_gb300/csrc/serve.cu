// Serving loop: continuous batching of encrypted KAN requests.
//
// Requests (one input ciphertext each, encrypted by their client) are
// admitted first-come first-served while the sum of their device-memory
// footprints stays within the HBM budget. A model's footprint per request is
// measured when the model is added: the whole network runs once on a zero
// ciphertext at the top level through the same per-layer path as a step, and
// the rise of the device memory pool's used-bytes watermark over what was in
// use before is recorded (the model's plaintext caches are filled by a first
// run that is not counted). A batch of B requests needs at most B times that:
// every buffer of the schedule grows with the batch. A request whose
// footprint exceeds the whole budget is refused at submission. Each step's
// measured rise of the watermark is kept, so the budget can be checked
// against what the device actually allocated.
//
// Each scheduling step evaluates one KAN layer for every active request:
// requests of the same model, at the same layer and the same level are
// concatenated into one batch and run through the layer together, then split
// back. A request that arrives while others are mid-network joins at the
// next step at its own layer 0, so work of requests at different stages
// overlaps step by step on the device. Batching never changes a ciphertext:
// every batch element is computed independently, word for word as when
// evaluated alone.
#include <deque>
#include <map>
#include <tuple>

#include "ops.h"

namespace ck {
Ct kan_eval_layer(kan_model& M, int layer, const ckks_keys& keys, const ckks_ct& x);
Ct kan_refresh_for_layer(kan_model& M, int layer, const ckks_keys& keys, Ct x);
int kan_num_layers(const kan_model& M);
int kan_layer_chunks(const kan_model& M, int layer);
int kan_total_depth(const kan_model& M);
int kan_input_depth(const kan_model& M);
}  // namespace ck

using namespace ck;

namespace {

// Used-bytes accounting of the device's default memory pool, the pool every
// stream-ordered allocation of the library comes from. The pool counts an
// allocation when it is requested on the host, so no synchronisation is needed.
struct PoolMeter {
  cudaMemPool_t pool = nullptr;
  explicit PoolMeter(int device) { CK_CUDA(cudaDeviceGetDefaultMemPool(&pool, device)); }
  uint64_t get(cudaMemPoolAttr a) const {
    uint64_t v = 0;
    CK_CUDA(cudaMemPoolGetAttribute(pool, a, &v));
    return v;
  }
  uint64_t used() const { return get(cudaMemPoolAttrUsedMemCurrent); }
  uint64_t high() const { return get(cudaMemPoolAttrUsedMemHigh); }
  void reset_high() const {
    uint64_t z = 0;  // the watermark restarts from the current use
    CK_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &z));
  }
};

struct Request {
  uint64_t id = 0;
  int model = 0;
  int layer = 0;
  size_t footprint = 0;
  Ct ct;
  bool done = false;
};

}  // namespace

struct kan_server {
  Ctx* ctx = nullptr;
  size_t budget = 0, in_use = 0, peak_in_use = 0;
  size_t measured_peak = 0;  // largest rise of the pool's used bytes over one step
  std::vector<std::pair<kan_model*, const ckks_keys*>> models;
  std::vector<size_t> footprint;  // per model: measured bytes per request
  std::deque<std::unique_ptr<Request>> waiting;
  std::map<uint64_t, std::unique_ptr<Request>> active;
  std::map<uint64_t, std::unique_ptr<Request>> finished;
  uint64_t next_id = 1;
  uint64_t steps = 0, batches = 0;
};

namespace {

void admit(kan_server& S) {
  while (!S.waiting.empty()) {
    Request& r = *S.waiting.front();
    if (S.in_use + r.footprint > S.budget) break;  // wait for memory (fits alone: checked at submit)
    S.in_use += r.footprint;
    S.peak_in_use = std::max(S.peak_in_use, S.in_use);
    const uint64_t id = r.id;
    S.active[id] = std::move(S.waiting.front());
    S.waiting.pop_front();
  }
}

// One layer of one batch of requests of a model: concatenate, evaluate,
// split back into per-request ciphertexts (the pieces replace the inputs).
void run_group(Ctx& c, kan_model& M, const ckks_keys& K, int layer, std::vector<Ct*>& cts) {
  std::vector<const ckks_ct*> parts;
  for (Ct* p : cts) parts.push_back(p->get());
  Ct in = parts.size() == 1 ? ct_copy(c, *parts[0]) : op_concat(c, parts);
  const int chunks = kan_layer_chunks(M, layer);
  // a model with a bootstrapping plan refreshes the group as kan_infer does
  in = kan_refresh_for_layer(M, layer, K, std::move(in));
  Ct out = kan_eval_layer(M, layer, K, *in);
  in.reset();
  const size_t per = out->words() / out->B;
  size_t off = 0;
  for (Ct* p : cts) {
    const size_t b = (*p)->B / chunks;  // a wide layer folds K chunk ciphertexts into one
    Ct piece = ct_alloc(c, b, out->level, out->scale);
    CK_CUDA(cudaMemcpyAsync(piece->d.p, out->d.u64() + off * per, b * per * 8,
                            cudaMemcpyDeviceToDevice, c.stream));
    off += b;
    *p = std::move(piece);
  }
}

// Bytes one request of model m needs beyond its input ciphertext, measured.
size_t measure_footprint(kan_server& S, int m) {
  Ctx& c = *S.ctx;
  kan_model& M = *S.models[m].first;
  const ckks_keys& K = *S.models[m].second;
  const PoolMeter pm(c.device);
  size_t need = 0;
  for (int pass = 0; pass < 2; pass++) {  // the first pass fills the plaintext caches
    Ct x = ct_alloc(c, (size_t)kan_layer_chunks(M, 0), c.L, c.delta[c.L]);
    CK_CUDA(cudaMemsetAsync(x->d.p, 0, x->d.bytes, c.stream));
    const uint64_t base = pm.used();
    pm.reset_high();
    std::vector<Ct*> one{&x};
    for (int layer = 0; layer < kan_num_layers(M); layer++) run_group(c, M, K, layer, one);
    need = (size_t)(pm.high() - base);
  }
  return need;
}

size_t step(kan_server& S) {
  const PoolMeter pm(S.ctx->device);
  const uint64_t base = pm.used();
  pm.reset_high();
  admit(S);
  // group by (model, layer, level)
  std::map<std::tuple<int, int, int>, std::vector<Request*>> groups;
  for (auto& kv : S.active) {
    Request* r = kv.second.get();
    groups[std::make_tuple(r->model, r->layer, r->ct->level)].push_back(r);
  }
  Ctx& c = *S.ctx;
  size_t completed = 0;
  for (auto& g : groups) {
    std::vector<Request*>& rs = g.second;
    kan_model& M = *S.models[std::get<0>(g.first)].first;
    const ckks_keys& K = *S.models[std::get<0>(g.first)].second;
    std::vector<Ct*> cts;
    for (Request* r : rs) cts.push_back(&r->ct);
    run_group(c, M, K, std::get<1>(g.first), cts);
    S.batches++;
    for (Request* r : rs) {
      r->layer++;
      if (r->layer == kan_num_layers(M)) r->done = true;
    }
  }
  S.measured_peak = std::max(S.measured_peak, (size_t)(pm.high() - base));
  for (auto it = S.active.begin(); it != S.active.end();) {
    if (it->second->done) {
      S.in_use -= it->second->footprint;
      S.finished[it->first] = std::move(it->second);
      it = S.active.erase(it);
      completed++;
    } else {
      ++it;
    }
  }
  S.steps++;
  return completed;
}

template <class F>
int guard(F&& f) {
  try {
    f();
    return CKKS_OK;
  } catch (...) {
    return api_error();
  }
}

}  // namespace

extern "C" {

int kan_server_create(ckks_ctx* ctx, size_t hbm_budget_bytes, kan_server** out) {
  return guard([&] {
    if (!ctx || !out || hbm_budget_bytes == 0) throw Error(CKKS_ERR_INVALID_ARG, "bad argument");
    auto s = std::make_unique<kan_server>();
    s->ctx = &ctx->c;
    s->budget = hbm_budget_bytes;
    *out = s.release();
  });
}

int kan_server_destroy(kan_server* s) {
  return guard([&] { delete s; });
}

int kan_server_add_model(kan_server* s, kan_model* model, const ckks_keys* keys, int* model_id) {
  return guard([&] {
    if (!s || !model || !keys || !model_id) throw Error(CKKS_ERR_INVALID_ARG, "bad argument");
    if (s->ctx->L < kan_input_depth(*model))
      throw Error(CKKS_ERR_LEVEL, "the model is deeper than the chain (and has no bootstrapping plan)");
    s->models.emplace_back(model, keys);
    const int m = (int)s->models.size() - 1;
    s->footprint.push_back(0);
    s->footprint[m] = measure_footprint(*s, m);
    *model_id = m;
  });
}

int kan_server_submit(kan_server* s, int model_id, const ckks_ct* in, uint64_t* request_id) {
  return guard([&] {
    if (!s || !in || !request_id || model_id < 0 || model_id >= (int)s->models.size())
      throw Error(CKKS_ERR_INVALID_ARG, "bad argument");
    if (in->level < kan_input_depth(*s->models[model_id].first))
      throw Error(CKKS_ERR_LEVEL, "input level below the model's depth");
    auto r = std::make_unique<Request>();
    r->id = s->next_id++;
    r->model = model_id;
    r->ct = ct_copy(*s->ctx, *in);
    r->footprint = s->footprint[model_id];
    if (r->footprint > s->budget) throw Error(CKKS_ERR_OUT_OF_MEMORY, "request exceeds the HBM budget");
    *request_id = r->id;
    s->waiting.push_back(std::move(r));
  });
}

int kan_server_step(kan_server* s, size_t* completed) {
  return guard([&] {
    if (!s) throw Error(CKKS_ERR_INVALID_ARG, "bad argument");
    const size_t n = step(*s);
    if (completed) *completed = n;
  });
}

int kan_server_take(kan_server* s, uint64_t request_id, ckks_ct** out) {
  if (!s || !out) return CKKS_ERR_INVALID_ARG;
  auto it = s->finished.find(request_id);
  if (it == s->finished.end()) {
    if (s->active.count(request_id)) return CKKS_PENDING;
    for (auto& w : s->waiting)
      if (w->id == request_id) return CKKS_PENDING;
    return CKKS_ERR_INVALID_ARG;
  }
  *out = it->second->ct.release();
  s->finished.erase(it);
  return CKKS_OK;
}

int kan_server_status(const kan_server* s, size_t* waiting, size_t* active, size_t* finished,
                      size_t* hbm_in_use, size_t* hbm_peak, size_t* hbm_measured_peak) {
  if (!s) return CKKS_ERR_INVALID_ARG;
  if (waiting) *waiting = s->waiting.size();
  if (active) *active = s->active.size();
  if (finished) *finished = s->finished.size();
  if (hbm_in_use) *hbm_in_use = s->in_use;
  if (hbm_peak) *hbm_peak = s->peak_in_use;
  if (hbm_measured_peak) *hbm_measured_peak = s->measured_peak;
  return CKKS_OK;
}

int kan_server_footprint(const kan_server* s, int model_id, size_t* bytes) {
  if (!s || !bytes || model_id < 0 || model_id >= (int)s->models.size()) return CKKS_ERR_INVALID_ARG;
  *bytes = s->footprint[model_id];
  return CKKS_OK;
}

}  // extern "C"
