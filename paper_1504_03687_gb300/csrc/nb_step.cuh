// nb_step.cuh — device-driven block steps (internal; not part of the ABI): the parameters of
// one block step in device memory, the step selection one warp runs, and the scheduler's
// device state.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

struct nb_sched;

namespace nbgpu {

// ---- device-driven block steps ------------------------------------------------------------
// The parameters of one block step held in device memory, so that a batch of block steps can
// be enqueued with no host work in between: the step's begin kernel (ac.cu) writes them from
// the scheduler's device state, and every later kernel of the step reads them.  A nonzero
// halt turns every kernel of the step, and of every step queued after it, into a no-op.
struct StepParams {
    double t;          // block time
    int64_t t_ticks;   // block time in ticks of 2^-48
    int64_t n_act;     // active particles: the list prefix [0, n_act)
    float t_hi, t_lo;  // the block time as a double-single pair
    int32_t lstar;     // coarsest active level
    int32_t halt;      // 0 run; 1 end time passed; 2 a regular step is due; 3 prefix too long; 4 batch done
};
enum { STEP_RUN = 0, STEP_END = 1, STEP_REGULAR = 2, STEP_LONG = 3, STEP_BUDGET = 4 };

// The begin of a device-driven block step (Sec. 3.3.1's block-step selection), one warp;
// lane l holds the counts of levels l and l + 32 and T is the current time in ticks.  The
// next block time is T + 2^-Lmax, Lmax the finest level present; its active particles are
// the levels >= L* = 48 - ctz(T_new), the list prefix of their total count.  The run halts
// when no particle is left, the time passes t_end, the budget is spent, the prefix is longer
// than max_prefix, or halt_hist (the regular-level histogram) holds a particle at a level
// >= L* (a regular step is due: the host takes it).  Otherwise P receives the step and the
// budget words are advanced: [0] steps left, [1] steps taken, [2] active rows taken.
struct StepBegin {
    StepParams *P;
    const int32_t *halt_hist;  // [64]
    double t_end;
    int64_t *budget;
    int64_t max_prefix;
};

// The inputs of step_begin that do not change during a device-driven step, read ahead.
struct StepBeginIn {
    int32_t r_lo, r_hi;  // halt_hist[lane], halt_hist[lane + 32]
    int64_t left;        // budget[0]
};
__device__ __forceinline__ StepBeginIn step_begin_inputs(const StepBegin &B, int lane)
{
    return StepBeginIn{B.halt_hist[lane], B.halt_hist[lane + 32], B.budget[0]};
}

__device__ __forceinline__ void step_begin(const StepBegin &B, int64_t c_lo, int64_t c_hi, int64_t T, int lane,
                                           const StepBeginIn &in)
{
    constexpr int kTicks = 48;
    const int32_t r_lo = in.r_lo, r_hi = in.r_hi;
    const int64_t left = in.left;
    StepParams *P = B.P;
    if (left <= 0) {
        if (lane == 0) P->halt = STEP_BUDGET;
        return;
    }
    const unsigned m_hi = __ballot_sync(0xffffffffu, c_hi != 0), m_lo = __ballot_sync(0xffffffffu, c_lo != 0);
    const int lmax = m_hi ? 63 - __clz(m_hi) : (m_lo ? 31 - __clz(m_lo) : -1);
    if (lmax < 0) {
        if (lane == 0) P->halt = STEP_END;
        return;
    }
    const int64_t T_new = T + ((int64_t)1 << (kTicks - lmax));
    const double t = ldexp((double)T_new, -kTicks);
    if (t > B.t_end) {
        if (lane == 0) P->halt = STEP_END;
        return;
    }
    int lstar = kTicks - (__ffsll(T_new) - 1);
    if (lstar < 0) lstar = 0;
    int64_t na = (lane >= lstar ? c_lo : 0) + (lane + 32 >= lstar ? c_hi : 0);
    int64_t nr = (lane >= lstar ? r_lo : 0) + (lane + 32 >= lstar ? r_hi : 0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        na += __shfl_xor_sync(0xffffffffu, na, o);
        nr += __shfl_xor_sync(0xffffffffu, nr, o);
    }
    if (lane != 0) return;
    if (nr > 0 || na > B.max_prefix) {
        P->halt = nr > 0 ? STEP_REGULAR : STEP_LONG;
        return;
    }
    P->t = t;
    P->t_ticks = T_new;
    P->n_act = na;
    P->lstar = lstar;
    P->t_hi = (float)t;
    P->t_lo = (float)(t - (double)P->t_hi);
    B.budget[0] = left - 1;
    B.budget[1] += 1;
    B.budget[2] += na;
}

// The scheduler's state on the device for device-driven steps (sched.cu): the list, device
// copies of the per-level counts and of the current time, and the longest prefix one device
// re-sort takes (one CTA).
struct SchedDevice {
    int32_t *list;
    int64_t *count;  // [64]
    int64_t *T;
    int64_t max_prefix;
};
bool sched_device(::nb_sched *s, SchedDevice *out);  // allocates the device copies on first use
bool sched_push(::nb_sched *s);                      // host counts and time -> device (stream-ordered)
bool sched_pull(::nb_sched *s);                      // device -> host (synchronises the stream)

}  // namespace nbgpu
