// internal.h -- library functions shared between its translation units, not exported.
#pragma once
#include <cstddef>
#include <cstdint>

#include "supra.h"

namespace supra {
// Workspace a batched B-mode call cannot run without: the frames' own parts (lines to
// scan-convert, the unfused chain of compounding frames).  supra_bmode_workspace_size adds
// the depth-segment boundary records, which the call uses when the workspace holds them.
size_t bmode_min_workspace(int32_t n, const supra_plan *const *plans);
}  // namespace supra
