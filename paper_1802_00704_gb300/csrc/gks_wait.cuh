// Bounded device-side wait on a flag written by another thread of the same
// launch (the sync-free triangular solves of the exact ILU preconditioner).
//
// The producer stores its data, executes __threadfence() and then stores the
// flag; the consumer waits until it sees the flag, executes __threadfence()
// and reads the data through L2 (__ldcg), so it sees the producer's stores.
// Every wait gives up after limit_ns nanoseconds of the GPU's global timer or
// as soon as another wait has given up (the shared error word err), so no
// launch can hang: a kernel that hits the limit sets err and finishes with
// unusable results, which the host learns from the status words.
#pragma once

#include <cstdint>

namespace gks {

// nanoseconds of the GPU's global timer (%globaltimer)
__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait until *flag == tag.  True once seen; false if the wait ran out (it then
// sets *err) or found *err already set.
__device__ __forceinline__ bool bounded_wait(const int32_t *flag, int32_t tag, int32_t *err, uint64_t limit_ns)
{
    const volatile int32_t *f = flag;
    if (*f != tag) {
        const volatile int32_t *e = err;
        const uint64_t t0 = global_ns();
        unsigned sleep = 32;
        for (unsigned n = 0; *f != tag; ++n) {
            if ((n & 15u) == 15u) {
                if (*e) return false;
                if (global_ns() - t0 > limit_ns) {
                    atomicExch(err, 1);
                    return false;
                }
            }
            __nanosleep(sleep);
            if (sleep < 128) sleep <<= 1;
        }
    }
    __threadfence();
    return true;
}

// Wait until *f[q] == tag for each of the three flags that is not NULL: their
// loads are issued together, so a row with several neighbours pays one round
// trip, not one per neighbour.  Same limits and error word as bounded_wait.
__device__ __forceinline__ bool bounded_wait_all(const int32_t *f0, const int32_t *f1, const int32_t *f2,
                                                 int32_t tag, int32_t *err, uint64_t limit_ns)
{
    auto ready = [&]() {
        const bool a = !f0 || *(const volatile int32_t *)f0 == tag;
        const bool b = !f1 || *(const volatile int32_t *)f1 == tag;
        const bool c = !f2 || *(const volatile int32_t *)f2 == tag;
        return a && b && c;
    };
    if (!ready()) {
        const volatile int32_t *e = err;
        const uint64_t t0 = global_ns();
        unsigned sleep = 32;
        for (unsigned c = 0; !ready(); ++c) {
            if ((c & 15u) == 15u) {
                if (*e) return false;
                if (global_ns() - t0 > limit_ns) {
                    atomicExch(err, 1);
                    return false;
                }
            }
            __nanosleep(sleep);
            if (sleep < 128) sleep <<= 1;
        }
    }
    __threadfence();
    return true;
}

// Publish: the caller's earlier stores become visible before the flag does.
__device__ __forceinline__ void publish(int32_t *flag, int32_t tag)
{
    __threadfence();
    *(volatile int32_t *)flag = tag;
}

}  // namespace gks
