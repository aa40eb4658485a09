// fk_streams.cu -- library-owned streams for running independent parts of one
// call concurrently: forked from the caller's stream by an event and joined
// back to it by events, so a call stays stream-ordered for its caller and
// capturable in a CUDA graph.  Three pools per device: the groups of the
// batched path, the parts inside one operation (which the batched path may
// itself run on a pooled stream), and the merge levels inside one of those
// parts.  Each pool's mutex is
// held by a call while it enqueues, so overlapping calls from several host
// threads do not interleave their fork and join events.
#include <mutex>

#include "fk_internal.cuh"

namespace fk {
namespace {

struct Pool {
    cudaStream_t s[kPoolStreams];
    cudaEvent_t fork;
    cudaEvent_t join[kPoolStreams];
    cudaEvent_t aux[kPoolAux];
    bool ready = false;
};
// Pool instances per device: a call forks onto the instance its own stream
// maps to, so operations issued from different streams fork onto different
// streams and can overlap.
constexpr int kSlots = 4;
std::mutex g_mu[kPools][kSlots];
Pool g_pool[kPools][64][kSlots];

int slot_of(cudaStream_t st) {
    const uintptr_t v = (uintptr_t)st;
    return (int)((v ^ (v >> 7) ^ (v >> 13)) % kSlots);
}

}  // namespace

fk_status StreamFork::begin(int which, cudaStream_t main, int k) {
    st = main;
    n = k < 1 ? 1 : (k > kPoolStreams ? kPoolStreams : k);
    s[0] = main;
    if (n == 1) return FK_OK;
    int dev = 0;
    FK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return set_error(FK_ERR_UNSUPPORTED, "device index %d", dev);
    pool = which;
    slot_ = slot_of(main);
    lock = std::unique_lock<std::mutex>(g_mu[which][slot_]);
    Pool& p = g_pool[which][dev][slot_];
    if (!p.ready) {
        for (int i = 1; i < kPoolStreams; ++i) FK_CUDA(cudaStreamCreateWithFlags(&p.s[i], cudaStreamNonBlocking));
        FK_CUDA(cudaEventCreateWithFlags(&p.fork, cudaEventDisableTiming));
        for (int i = 1; i < kPoolStreams; ++i) FK_CUDA(cudaEventCreateWithFlags(&p.join[i], cudaEventDisableTiming));
        for (int i = 0; i < kPoolAux; ++i) FK_CUDA(cudaEventCreateWithFlags(&p.aux[i], cudaEventDisableTiming));
        p.ready = true;
    }
    dev_ = dev;
    for (int i = 0; i < kPoolAux; ++i) ev[i] = p.aux[i];
    FK_CUDA(cudaEventRecord(p.fork, main));
    for (int i = 1; i < n; ++i) {
        s[i] = p.s[i];
        FK_CUDA(cudaStreamWaitEvent(p.s[i], p.fork, 0));
    }
    forked = true;
    return FK_OK;
}

fk_status StreamFork::end() {
    if (!forked) return FK_OK;
    forked = false;
    Pool& p = g_pool[pool][dev_][slot_];
    fk_status rc = FK_OK;
    for (int i = 1; i < n; ++i) {
        const cudaError_t e1 = cudaEventRecord(p.join[i], p.s[i]);
        const cudaError_t e2 = cudaStreamWaitEvent(st, p.join[i], 0);
        if (rc == FK_OK && (e1 != cudaSuccess || e2 != cudaSuccess))
            rc = cuda_error(e1 != cudaSuccess ? e1 : e2, "stream join");
    }
    if (lock.owns_lock()) lock.unlock();
    return rc;
}

StreamFork::~StreamFork() { end(); }

}  // namespace fk
