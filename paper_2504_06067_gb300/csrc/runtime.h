// runtime.h -- host-side pieces shared by the context engine (engine.cu) and
// the run server (server.cu): a device-memory arena and the internal forms of
// context creation / destruction.  Not part of the C ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <map>
#include <mutex>
#include <string>

#include "nsga3.h"

// One cudaMalloc of a fixed budget, handed out in 256-byte-aligned blocks by
// first fit over a free list ordered by offset (neighbours coalesce on
// release).  Thread-safe.  Releasing never synchronises the device: the
// caller must know that no queued work still uses the block.
class DeviceArena {
public:
    static constexpr size_t kAlign = 256;

    // Takes ownership of [base, base + bytes).
    DeviceArena(void* base, size_t bytes);
    void* alloc(size_t bytes);     // nullptr when no free block is large enough
    void release(void* p);         // p must come from alloc()
    size_t capacity() const { return cap_; }
    size_t in_use() const;
    size_t largest_free() const;
    void* base() const { return base_; }

    static size_t round_up(size_t b) { return (b + kAlign - 1) / kAlign * kAlign; }

private:
    char* base_;
    size_t cap_;
    size_t used_ = 0;
    std::map<size_t, size_t> free_;  // offset -> size
    std::map<size_t, size_t> live_;  // offset -> size
    mutable std::mutex mu_;
};

// Context creation with optional arena (nullptr: cudaMalloc per buffer).
// shared_gpu: the run will share the GPU with other runs (its cooperative
// launches take fewer CTAs).  On failure *err holds the message and *out is
// nullptr.
nsga3_status ctx_create(int m, int d, int N, int ref_divisions, const nsga3_opts* opts, DeviceArena* arena,
                        nsga3_ctx** out, std::string* err, bool shared_gpu = false);

// Device bytes ctx_create allocates for these arguments (each buffer rounded
// up to DeviceArena::kAlign), computed without touching the device when
// `num_sms` > 0 is given.
nsga3_status ctx_workspace_bytes(int m, int d, int N, int ref_divisions, const nsga3_opts* opts, int num_sms,
                                 size_t* bytes, std::string* err);

// Destroys a context.  sync_device = false skips the device-wide
// synchronisation of nsga3_destroy: the caller guarantees that the
// context's work has completed (e.g. its stream was synchronised).
void ctx_destroy(nsga3_ctx* ctx, bool sync_device);

// Kernel launches made for ctx so far (as nsga3_total_launches), reading the
// device counter on `stream` and synchronising only that stream.
nsga3_status ctx_launches(nsga3_ctx* ctx, void* stream, long long* launches);
