// Host-side helpers: device buffers and error propagation.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <map>
#include <string>
#include <vector>

namespace bddc {

struct Error {
    int status;
    std::string msg;
};

#define BDDC_CUDA(call)                                                                         \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            throw ::bddc::Error{7, std::string(#call) + ": " + cudaGetErrorString(e_)};         \
    } while (0)

#define BDDC_REQUIRE(cond, status, msg)                                                         \
    do {                                                                                        \
        if (!(cond)) throw ::bddc::Error{(status), (msg)};                                      \
    } while (0)

// Named device allocations that keep their capacity across repeated phases.
// Memory comes from cudaMalloc, or from the caller's allocator when one is set
// (set_allocator); the caller's free receives the pointer and its size.
class Arena {
  public:
    using AllocFn = void *(*)(size_t bytes, void *ctx);
    using FreeFn = void (*)(void *ptr, size_t bytes, void *ctx);
    ~Arena() { release(); }
    void set_allocator(AllocFn a, FreeFn f, void *ctx, cudaStream_t stream) {
        alloc_ = a;
        free_ = f;
        ctx_ = ctx;
        stream_ = stream;
    }
    void *get(const std::string &name, size_t bytes) {
        if (bytes == 0) bytes = 16;
        auto it = bufs_.find(name);
        if (it != bufs_.end() && it->second.second >= bytes) return it->second.first;
        if (it != bufs_.end()) {
            dev_free(it->second.first, it->second.second);
            total_ -= it->second.second;
            bufs_.erase(it);
        }
        void *p = nullptr;
        if (alloc_) {
            p = alloc_(bytes, ctx_);
            if (!p) throw Error{2, "allocator callback returned NULL for " + name + " (" + std::to_string(bytes) + " bytes)"};
        } else {
            cudaError_t e = cudaMalloc(&p, bytes);
            if (e != cudaSuccess)
                throw Error{2, "cudaMalloc(" + name + ", " + std::to_string(bytes) + "): " + cudaGetErrorString(e)};
        }
        bufs_[name] = {p, bytes};
        total_ += bytes;
        return p;
    }
    template <typename T>
    T *get_t(const std::string &name, size_t count) {
        return static_cast<T *>(get(name, count * sizeof(T)));
    }
    template <typename T>
    T *upload(const std::string &name, const std::vector<T> &v, cudaStream_t s) {
        T *p = get_t<T>(name, v.size());
        if (!v.empty()) {
            cudaError_t e = cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) throw Error{7, "upload " + name + ": " + cudaGetErrorString(e)};
        }
        return p;
    }
    void release() {
        for (auto &kv : bufs_) dev_free(kv.second.first, kv.second.second);
        bufs_.clear();
        total_ = 0;
    }
    size_t total() const { return total_; }

  private:
    void dev_free(void *p, size_t bytes) {
        if (free_) {
            // work queued on the stream may still read the buffer
            cudaStreamSynchronize(stream_);
            free_(p, bytes, ctx_);
        } else {
            cudaFree(p);
        }
    }
    std::map<std::string, std::pair<void *, size_t>> bufs_;
    size_t total_ = 0;
    AllocFn alloc_ = nullptr;
    FreeFn free_ = nullptr;
    void *ctx_ = nullptr;
    cudaStream_t stream_ = nullptr;
};

}  // namespace bddc
