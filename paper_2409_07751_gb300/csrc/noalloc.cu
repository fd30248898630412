// Allocation-free rescale for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocating routine) at the
// point where they rescale: code running while a CUDA stream is being
// captured into a graph, runtimes that hand out a fixed device-memory budget
// up front, or real-time loops that forbid allocator calls. For them this
// file keeps the rescale's working memory (the copied top limb and the
// spread correction term) in one file-scope device array of fixed size
// instead of asking an allocator for it. The caller still passes the input
// and output ciphertext memory.
//
// The array is sized for 8 Mi words (64 MiB); every GPU that loads this
// library holds it until the process exits. Its address is looked up once
// per device on the first call (with that device current), so the first call
// on each device should happen before any stream capture. All calls share
// the array: two calls that overlap on the GPU (different streams, or
// different host threads) race on it and must be serialized by the caller.
// Both scratch regions are fully written before they are read, so nothing
// in the array needs clearing between calls.
#include <mutex>

#include "ops.h"

using namespace ck;

namespace {

constexpr size_t NOALLOC_SCRATCH_WORDS = (size_t)8 << 20;
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) uint64_t g_noalloc_scratch[NOALLOC_SCRATCH_WORDS];

std::mutex g_mu;
uint64_t* g_scratch_addr[MAX_DEVICES] = {};

// Device address of the scratch array on `device` (host code must not use
// the array's name as a device pointer).
uint64_t* scratch_on(int device) {
  if (device < 0 || device >= MAX_DEVICES) throw Error(CKKS_ERR_UNSUPPORTED, "device ordinal >= 64");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    CK_CUDA(cudaSetDevice(device));
    CK_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_scratch_addr[device] = static_cast<uint64_t*>(p);
  }
  return g_scratch_addr[device];
}

}  // namespace

extern "C" int ckks_rescale_noalloc(ckks_ctx* ctx, const uint64_t* d_in, size_t batch, int level,
                                    uint64_t* d_out) {
  try {
    if (!ctx || !d_in || !d_out || batch == 0) return CKKS_ERR_INVALID_ARG;
    Ctx& c = ctx->c;
    if (level < 1 || level > c.L) return CKKS_ERR_LEVEL;
    const size_t polys = 2 * batch;
    const size_t need = polys * c.N * (size_t)(1 + level);
    if (need > NOALLOC_SCRATCH_WORDS) return CKKS_ERR_INVALID_ARG;
    CK_CUDA(cudaSetDevice(c.device));
    uint64_t* last = scratch_on(c.device);
    uint64_t* R = last + polys * c.N;
    CK_CUDA(cudaMemcpy2DAsync(last, c.N * 8, d_in + (size_t)level * c.N,
                              (size_t)(level + 1) * c.N * 8, c.N * 8, polys,
                              cudaMemcpyDeviceToDevice, c.stream));
    ntt_inverse(c, last, polys, c.iota() + level, 1);
    k_rescale_spread(c, last, R, polys, level);
    ntt_forward(c, R, polys * level, c.iota(), level);
    k_rescale_finish(c, d_in, R, d_out, polys, level, c.d_rs_inv.u64() + (size_t)level * (c.L + 1),
                     c.d_rs_invs.u64() + (size_t)level * (c.L + 1));
    return CKKS_OK;
  } catch (...) {
    return api_error();
  }
}
