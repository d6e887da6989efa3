// The single-CTA path's launcher with a choice of block size (sssp_small.cu).
#pragma once

#include "bfq_internal.h"

namespace bfq {

// The run on one CTA of `threads` threads (512 or 1024): fewer warps contend
// for the ring on deep, narrow searches, more keep up on denser graphs.
// Kernel bracketed by ev0/ev1 when given, then the epilogue.
cudaError_t launch_sssp_small_threads(const SsspArgs& a, int cap_log2, int threads,
                                      int32_t* status_dev, cudaEvent_t ev0, cudaEvent_t ev1,
                                      cudaStream_t s);

}  // namespace bfq
