// Error handling, launch accounting and memory helpers.
#include <cstring>
#include <map>
#include <mutex>
#include <unordered_map>

#include "common.h"

namespace h2 {

std::atomic<int64_t> g_launches{0};

void fail(int status, const std::string& msg) { throw Error(status, msg); }

void check_cuda(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        fail(H2_ERR_OOM, std::string(what) + ": " + cudaGetErrorString(e));
    }
    fail(H2_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void after_launch(const char* name) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) fail(H2_ERR_CUDA, std::string("launch of ") + name + ": " + cudaGetErrorString(e));
}

namespace {

// Kept blocks of one kind (device or pinned host), by size.
struct FreeList {
    std::multimap<size_t, void*> blocks;
    size_t bytes = 0;
    // smallest kept block of at least `want` bytes and at most twice that (plus 64 KB)
    void* take(size_t want, size_t* got) {
        auto it = blocks.lower_bound(want);
        if (it == blocks.end() || it->first > 2 * want + (size_t(64) << 10)) return nullptr;
        void* p = it->second;
        *got = it->first;
        bytes -= it->first;
        blocks.erase(it);
        return p;
    }
};

struct ThreadCache {
    cudaStream_t s = nullptr;
    std::unordered_map<void*, size_t> dev_live, host_live;   // blocks allocated inside the scope
    FreeList dev_kept, host_kept;
};

constexpr size_t kDevKeepMax = size_t(16) << 30;    // kept device bytes per thread
constexpr size_t kHostKeepMax = size_t(512) << 20;  // kept pinned bytes per thread

thread_local ThreadCache* t_cache = nullptr;

// round up by at most a quarter: multiples of max(4 KB, 2^(floor(log2 b) - 2))
size_t size_class(size_t b) {
    size_t g = 4096;
    while (g * 8 <= b) g <<= 1;
    return (b + g - 1) / g * g;
}

// Accounting of the library's device blocks (all threads): live bytes, and an optional cap that
// turns any allocation above it into H2_ERR_OOM (allocation-failure tests without exhausting the
// device).
std::mutex g_dev_mu;
std::unordered_map<void*, size_t> g_dev_sizes;
int64_t g_dev_live = 0, g_dev_limit = 0;

void* raw_dev_alloc(size_t bytes) {
    std::lock_guard<std::mutex> lock(g_dev_mu);
    if (g_dev_limit > 0 && g_dev_live + (int64_t)bytes > g_dev_limit)
        fail(H2_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes above the library's limit of " +
                             std::to_string(g_dev_limit) + " bytes");
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(H2_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e));
    }
    g_dev_sizes[p] = bytes;
    g_dev_live += (int64_t)bytes;
    return p;
}

void raw_dev_free(void* p) {
    {
        std::lock_guard<std::mutex> lock(g_dev_mu);
        auto it = g_dev_sizes.find(p);
        if (it != g_dev_sizes.end()) {
            g_dev_live -= (int64_t)it->second;
            g_dev_sizes.erase(it);
        }
    }
    cudaFree(p);
}

void* raw_host_alloc(size_t bytes) {
    void* p = nullptr;
    cudaError_t e = cudaMallocHost(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(H2_ERR_OOM, "cudaMallocHost of " + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e));
    }
    return p;
}

template <class RawAlloc>
void* cached_alloc(size_t bytes, FreeList& kept, std::unordered_map<void*, size_t>& live, RawAlloc raw) {
    const size_t want = size_class(bytes);
    size_t got = 0;
    void* p = kept.take(want, &got);
    if (!p) {
        p = raw(want);
        got = want;
    }
    live[p] = got;
    return p;
}

// true if the block was kept for reuse
bool cached_free(void* p, FreeList& kept, std::unordered_map<void*, size_t>& live, size_t keep_max) {
    auto it = live.find(p);
    if (it == live.end()) return false;
    const size_t sz = it->second;
    live.erase(it);
    if (kept.bytes + sz > keep_max) return false;
    kept.blocks.emplace(sz, p);
    kept.bytes += sz;
    return true;
}

}  // namespace

void* dev_alloc_bytes(size_t bytes) {
    if (t_cache) return cached_alloc(bytes, t_cache->dev_kept, t_cache->dev_live, raw_dev_alloc);
    return raw_dev_alloc(bytes);
}

void dev_free(void* p) {
    if (!p) return;
    if (t_cache && cached_free(p, t_cache->dev_kept, t_cache->dev_live, kDevKeepMax)) return;
    raw_dev_free(p);
}

void* host_alloc_bytes(size_t bytes) {
    if (t_cache) return cached_alloc(bytes, t_cache->host_kept, t_cache->host_live, raw_host_alloc);
    return raw_host_alloc(bytes);
}

void host_free(void* p) {
    if (!p) return;
    if (t_cache && cached_free(p, t_cache->host_kept, t_cache->host_live, kHostKeepMax)) return;
    cudaFreeHost(p);
}

void dev_alloc_limit(int64_t bytes) {
    std::lock_guard<std::mutex> lock(g_dev_mu);
    g_dev_limit = bytes > 0 ? bytes : 0;
}

int64_t dev_live_bytes() {
    std::lock_guard<std::mutex> lock(g_dev_mu);
    return g_dev_live;
}

AllocScope::AllocScope(cudaStream_t s) {
    if (t_cache) return;
    t_cache = new ThreadCache();
    t_cache->s = s;
    owner_ = true;
}

AllocScope::~AllocScope() {
    if (!owner_) return;
    ThreadCache* c = t_cache;
    t_cache = nullptr;
    cudaStreamSynchronize(c->s);
    for (auto& b : c->dev_kept.blocks) raw_dev_free(b.second);
    for (auto& b : c->host_kept.blocks) cudaFreeHost(b.second);
    delete c;
}

Stager::~Stager() {
    if (ev) {
        cudaEventSynchronize(ev);
        cudaEventDestroy(ev);
    }
    host_free(host);
}

void Stager::copy(void* dst, const void* src, size_t bytes, cudaStream_t s) {
    if (!ev) H2_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    H2_CUDA(cudaEventSynchronize(ev));  // previous copy out of the buffer has finished
    if (bytes > cap) {
        host_free(host);
        host = nullptr;
        cap = 0;
        size_t want = bytes < 4096 ? 4096 : bytes * 3 / 2;
        host = host_alloc_bytes(want);
        cap = want;
    }
    std::memcpy(host, src, bytes);
    H2_CUDA(cudaMemcpyAsync(dst, host, bytes, cudaMemcpyHostToDevice, s));
    H2_CUDA(cudaEventRecord(ev, s));
}

}  // namespace h2
