// Device-side bounds checks of index tables (validate.cu), for dfmm_validate.
#pragma once
#include <cstdint>
#include <vector>

#include "common.h"

namespace dfmm {

enum CheckMode {
  kCheckFields = 0,   // int32 entries of `stride` fields: field a in [0, hi_a); if b >= 0,
                      //   field b >= 0 and field a + field b <= hi_ab
  kCheckCsr32 = 1,    // int32 offsets [n + 1]: nondecreasing from 0 to hi_a
  kCheckCsr64 = 2,    // int64 offsets [n + 1]: likewise
  kCheckPacked = 3,   // uint32 words whose low 25 bits must be < hi_a
};

struct RangeCheck {
  const void* p = nullptr;   // device table
  int64_t n = 0;             // entries (offsets: n + 1 values)
  int mode = kCheckFields;
  int stride = 1, a = 0, b = -1;
  int64_t hi_a = 0, hi_ab = 0;
};

// Runs every check on `s` and synchronises; per check, the first entry out of
// range, or -1.
std::vector<int64_t> run_range_checks(const std::vector<RangeCheck>& checks, cudaStream_t s);

}  // namespace dfmm
