// Serving loop: continuous batching of encrypted KAN requests.
//
// Requests (one input ciphertext each, encrypted by their client) are
// admitted first-come first-served while the sum of their device-memory
// footprints stays within the HBM budget. Each scheduling step evaluates one
// KAN layer for every active request: requests of the same model, at the
// same layer and the same level are concatenated into one batch and run
// through the layer together, then split back. A request that arrives while
// others are mid-network joins at the next step at its own layer 0, so work
// of requests at different stages overlaps step by step on the device.
// Batching never changes a ciphertext: every batch element is computed
// independently, word for word as when evaluated alone.
#include <deque>
#include <map>
#include <tuple>

#include "ops.h"

namespace ck {
Ct kan_eval_layer(kan_model& M, int layer, const ckks_keys& keys, const ckks_ct& x);
int kan_num_layers(const kan_model& M);
int kan_layer_chunks(const kan_model& M, int layer);
int kan_total_depth(const kan_model& M);
}  // namespace ck

using namespace ck;

namespace {

// working set of one request while its layers run: the ciphertext plus the
// key-switching extension (about beta*(l+alpha) limbs) and the schedule's
// live temporaries, bounded here by 32 ciphertexts of the input's size
constexpr double FOOTPRINT_FACTOR = 32.0;

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
  std::vector<std::pair<kan_model*, const ckks_keys*>> models;
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
    if (S.in_use + r.footprint > S.budget && !S.active.empty()) break;  // wait for memory
    S.in_use += r.footprint;
    S.peak_in_use = std::max(S.peak_in_use, S.in_use);
    const uint64_t id = r.id;
    S.active[id] = std::move(S.waiting.front());
    S.waiting.pop_front();
  }
}

size_t step(kan_server& S) {
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
    std::vector<const ckks_ct*> parts;
    for (Request* r : rs) parts.push_back(r->ct.get());
    Ct in = parts.size() == 1 ? ct_copy(c, *parts[0]) : op_concat(c, parts);
    const int chunks = kan_layer_chunks(M, std::get<1>(g.first));
    Ct out = kan_eval_layer(M, std::get<1>(g.first), K, *in);
    S.batches++;
    const size_t per = out->words() / out->B;
    size_t off = 0;
    for (Request* r : rs) {
      const size_t b = r->ct->B / chunks;  // a wide layer folds K chunk ciphertexts into one
      Ct piece = ct_alloc(c, b, out->level, out->scale);
      CK_CUDA(cudaMemcpyAsync(piece->d.p, out->d.u64() + off * per, b * per * 8,
                              cudaMemcpyDeviceToDevice, c.stream));
      off += b;
      r->ct = std::move(piece);
      r->layer++;
      if (r->layer == kan_num_layers(M)) r->done = true;
    }
  }
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
    s->models.emplace_back(model, keys);
    *model_id = (int)s->models.size() - 1;
  });
}

int kan_server_submit(kan_server* s, int model_id, const ckks_ct* in, uint64_t* request_id) {
  return guard([&] {
    if (!s || !in || !request_id || model_id < 0 || model_id >= (int)s->models.size())
      throw Error(CKKS_ERR_INVALID_ARG, "bad argument");
    if (in->level < kan_total_depth(*s->models[model_id].first))
      throw Error(CKKS_ERR_LEVEL, "input level below the model's depth");
    auto r = std::make_unique<Request>();
    r->id = s->next_id++;
    r->model = model_id;
    r->ct = ct_copy(*s->ctx, *in);
    r->footprint = (size_t)(FOOTPRINT_FACTOR * (double)r->ct->d.bytes);
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
                      size_t* hbm_in_use, size_t* hbm_peak) {
  if (!s) return CKKS_ERR_INVALID_ARG;
  if (waiting) *waiting = s->waiting.size();
  if (active) *active = s->active.size();
  if (finished) *finished = s->finished.size();
  if (hbm_in_use) *hbm_in_use = s->in_use;
  if (hbm_peak) *hbm_peak = s->peak_in_use;
  return CKKS_OK;
}

}  // extern "C"
