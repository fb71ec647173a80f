// Admission policy of the request server (host logic only, no CUDA): which
// queued request runs next when a slot is free.  Requests are taken in
// arrival order; while the oldest one does not fit the free device budget,
// the first later request that fits may run ahead of it (backfilling), but
// at most max_bypass times per oldest request, after which that request is
// reserved: nothing passes it and it runs as soon as enough memory is free.
// The bound keeps a large request from starving behind a stream of small
// ones.
#pragma once

#include <cstdint>
#include <cstddef>

namespace sip {

// queue: a sequence of requests in arrival order, each with members `bytes`
// (its device footprint) and `bypassed` (how often a later request was
// admitted while it was the oldest).  Returns the index to admit, or -1.
// The caller increments queue[0].bypassed when the index is above 0.
template <class Queue>
int admission_pick(const Queue& queue, int64_t in_use, int64_t budget, int max_bypass) {
    if (queue.empty()) return -1;
    if (in_use + queue.front().bytes <= budget) return 0;
    if (queue.front().bypassed >= max_bypass) return -1;   // reserved: wait for memory
    for (std::size_t i = 1; i < queue.size(); ++i)
        if (in_use + queue[i].bytes <= budget) return int(i);
    return -1;
}

}  // namespace sip
