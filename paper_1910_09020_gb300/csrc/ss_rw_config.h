// ss_rw_config.h -- limits and launch shape of the plain kernels.
#pragma once

namespace ssk {

// Largest E and m served by the thread-per-pair row-wise kernel (K3a).
constexpr int kRwMaxE = 31;
constexpr int kRwMaxM = 1024;
constexpr int kRwThreads = 128;  // threads (= pairs) per tile

// Thresholds that may share one pass over the bit-sliced layout (0..4).
constexpr int kSlicedSetMaxE = 4;

}  // namespace ssk
