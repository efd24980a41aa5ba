// Error handling, launch accounting and memory helpers.
#include <cstring>

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

void* dev_alloc_bytes(size_t bytes) {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(H2_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e));
    }
    return p;
}

Stager::~Stager() {
    if (ev) {
        cudaEventSynchronize(ev);
        cudaEventDestroy(ev);
    }
    if (host) cudaFreeHost(host);
}

void Stager::copy(void* dst, const void* src, size_t bytes, cudaStream_t s) {
    if (!ev) H2_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    H2_CUDA(cudaEventSynchronize(ev));  // previous copy out of the buffer has finished
    if (bytes > cap) {
        if (host) cudaFreeHost(host);
        host = nullptr;
        cap = 0;
        size_t want = bytes < 4096 ? 4096 : bytes * 3 / 2;
        H2_CUDA(cudaMallocHost(&host, want));
        cap = want;
    }
    std::memcpy(host, src, bytes);
    H2_CUDA(cudaMemcpyAsync(dst, host, bytes, cudaMemcpyHostToDevice, s));
    H2_CUDA(cudaEventRecord(ev, s));
}

}  // namespace h2
