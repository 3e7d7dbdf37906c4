// Device memory of one library object (forest, batch, net): taken from the caller's allocator
// hook when one was given at creation, else from cudaMalloc / cudaFree.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <unordered_map>

#include "lbm_gb300.h"

namespace lbm {

class DevMem {
public:
    // Binds the hook (NULL or a hook without alloc: the CUDA runtime) and the stream the object
    // orders its work on.  Returns false if the hook has alloc but no release.
    bool bind(const lbm_allocator* hook, cudaStream_t stream) {
        stream_ = stream;
        if (hook && hook->alloc) {
            if (!hook->release) return false;
            hook_ = *hook;
        }
        return true;
    }

    bool hooked() const { return hook_.alloc != nullptr; }

    // `bytes` of device memory into *p (0 bytes: NULL).  False if the allocation failed or the hook
    // returned a pointer that is not 256-byte aligned (which is handed back at once).  Through a
    // hook, returns once the object's stream has finished the work queued on it.
    template <typename T>
    bool get(T** p, size_t bytes) {
        void* v = nullptr;
        const bool ok = get_raw(&v, bytes);
        *p = static_cast<T*>(v);
        return ok;
    }

    // Frees what get() returned (NULL: no-op).  Through a hook the memory is released only after
    // the object's stream has finished the work queued on it, since a caching allocator may hand
    // it out again at once.
    void put(const void* cp) {
        void* p = const_cast<void*>(cp);
        if (!p) return;
        if (!hooked()) {
            cudaFree(p);
            return;
        }
        auto it = sizes_.find(p);
        const size_t bytes = it == sizes_.end() ? 0 : it->second;
        if (it != sizes_.end()) sizes_.erase(it);
        cudaStreamSynchronize(stream_);
        hook_.release(p, bytes, stream_, hook_.user);
    }

    // Bytes currently held through the hook (0 without one).
    size_t held() const {
        size_t n = 0;
        for (const auto& kv : sizes_) n += kv.second;
        return n;
    }

private:
    bool get_raw(void** p, size_t bytes) {
        *p = nullptr;
        if (bytes == 0) return true;
        if (!hooked()) return cudaMalloc(p, bytes) == cudaSuccess;
        void* v = hook_.alloc(bytes, stream_, hook_.user);
        if (!v) return false;
        if (reinterpret_cast<uintptr_t>(v) % 256 != 0) {
            hook_.release(v, bytes, stream_, hook_.user);
            return false;
        }
        sizes_[v] = bytes;
        *p = v;
        // a caching allocator may hand out memory that work still queued on the stream uses; the
        // library fills new buffers with copies outside that stream, so let that work finish
        cudaStreamSynchronize(stream_);
        return true;
    }

    lbm_allocator hook_{};
    cudaStream_t stream_ = nullptr;
    std::unordered_map<void*, size_t> sizes_;
};

}  // namespace lbm
