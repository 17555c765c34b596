// Launch-sequence replay shared by the single and the batched sort.  A sort's
// launches depend only on its arguments and options (every grid is sized on
// the host, every data-dependent quantity stays on the device), so the
// sequence of a call can be captured into a CUDA graph once and replayed by
// later calls with the same key.
#pragma once

#include <array>
#include <cstdint>
#include <functional>

#include <cuda_runtime.h>

namespace pgs {

// Everything that shapes a call's launch sequence: the call kind, pointers,
// sizes, options and device.  Unused entries stay 0.
using GraphKey = std::array<uint64_t, 28>;

inline uint64_t key_ptr(const void* p) { return (uint64_t)reinterpret_cast<uintptr_t>(p); }

// Issues the call through the process-wide graph cache (16 keys, least
// recently used out).  The first call with a key runs `run(st)` directly and
// records the key; the second captures `run` on a stream of the library's own
// (thread-local capture mode), instantiates the graph and launches it on `st`;
// later calls launch that graph.  With `allow` false (a timer, the OFF option,
// a tuner's timed call), on a stream that is being captured, or for a key whose
// capture failed, `run(st)` runs directly.  `run` must issue every launch of
// the call on the stream it is given, never synchronise, and return a status.
int launch_cached(const GraphKey& key, bool allow, cudaStream_t st, const std::function<int(cudaStream_t)>& run);

}  // namespace pgs
