// Entry points shared between translation units of the library (not part of
// the C ABI).
#pragma once
#include <cstddef>

#include "dfmm.h"

namespace dfmm {

// Records `msg` as the calling thread's last error and returns `code`.
int set_error(int code, const char* msg);

// Server requests hold their plan: plan_acquire returns false for a handle that
// is not a live plan, else counts one holder (dfmm_destroy refuses a plan with
// holders); plan_release drops one.
bool plan_acquire(const dfmm_plan_s* plan);
void plan_release(const dfmm_plan_s* plan);

// The matvec of dfmm_apply with every per-apply buffer (states, staging
// buffers, work tiles) laid out inside the caller-provided device memory
// [scratch, scratch + bytes); no device memory is allocated.
int apply_with_scratch(dfmm_plan_s* plan, const void* f, void* u, int nrhs, cudaStream_t stream, void* scratch,
                       size_t bytes);

// Device address of the status word of the last allocation-free apply on the
// current device (offset 0 of its scratch array) if that apply was issued on
// `stream`, else nullptr.
const unsigned* noalloc_status_word(cudaStream_t stream);

}  // namespace dfmm
