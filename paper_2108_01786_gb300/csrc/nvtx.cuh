// NVTX ranges around the library's entry points and phases (visible in Nsight
// Systems / Compute timelines; no cost without a tool attached).
#pragma once
#include <nvtx3/nvToolsExt.h>

struct BieNvtxRange {
  explicit BieNvtxRange(const char* name) { nvtxRangePushA(name); }
  ~BieNvtxRange() { nvtxRangePop(); }
  BieNvtxRange(const BieNvtxRange&) = delete;
  BieNvtxRange& operator=(const BieNvtxRange&) = delete;
};
#define BIE_NVTX_CAT2(a, b) a##b
#define BIE_NVTX_CAT(a, b) BIE_NVTX_CAT2(a, b)
#define BIE_NVTX(name) BieNvtxRange BIE_NVTX_CAT(bie_nvtx_, __LINE__)(name)
