// NVTX ranges around the library's host entry points, so that a profiling session can attribute each kernel to
// the call that launched it (for example ncu --nvtx --nvtx-include "aim_batch_run/").  NVTX v3 is header-only;
// with no tool attached a push or pop only tests a function pointer.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace aim {

class Range {
public:
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

}  // namespace aim
