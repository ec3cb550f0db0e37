// sha3_queue_staged.cu -- the instances of the queue kernel (queue.cuh) with
// the looped permutation: direct loads, the next block copied into shared
// memory (cp.async), or the next block loaded into registers; compiled apart
// from the host logic of sha3_queue.cu so the two build in parallel.
//
// A block of 128 threads of the shared-memory form holds 2 x 43 x 128 words
// (44,032 bytes) of stages, so register budgets up to 4 blocks per SM are
// compiled; the register form keeps 43 more words live across the
// permutation, which fits the budgets of 2 and 3 blocks per SM without
// spilling.
#include <cuda_runtime.h>

#include "queue.cuh"

namespace kb {

#define KB_Q(M, S) reinterpret_cast<const void *>(&k_sha3_queue<M, S>)
const void *queue_kernel_staged(int minb, int stage) {
    switch (stage) {
        case kStageDirect | kLooped:
            return minb == 2 ? KB_Q(2, kLooped) : minb == 3 ? KB_Q(3, kLooped) : minb == 4 ? KB_Q(4, kLooped) : nullptr;
        case kStageAsync | kLooped:
            return minb == 2 ? KB_Q(2, kStageAsync | kLooped) : minb == 3 ? KB_Q(3, kStageAsync | kLooped)
                 : minb == 4 ? KB_Q(4, kStageAsync | kLooped) : nullptr;
        case kStageRegs | kLooped:
            return minb == 2 ? KB_Q(2, kStageRegs | kLooped) : minb == 3 ? KB_Q(3, kStageRegs | kLooped) : nullptr;
        default:
            return nullptr;
    }
}
#undef KB_Q

}  // namespace kb
