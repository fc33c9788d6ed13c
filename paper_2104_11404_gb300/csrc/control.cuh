// Automatic time-step control of Section 2.2.3 as device functions on one
// control block, shared by the single-instance step (one control block per
// context) and the batched step (one per instance).
#pragma once

#include "device_util.cuh"

namespace lagh {

constexpr unsigned long long kInfBits = 0x7ff0000000000000ull;

__device__ __forceinline__ double bits_to_tau(unsigned long long b) {
  return __longlong_as_double((long long)b);
}

struct CtlConsts {
  double beta1, beta2, gamma_dt;
};

// End of one attempt: redo with beta1 dt if dt >= tau (tau = the smaller of
// the two stage estimates; an inverted element counts as tau = 0), otherwise
// accept and grow by beta2 when dt <= gamma tau.  Prepares dt_use for the next
// attempt (clamped to land on t_final) and resets the per-stage estimates.
__device__ __forceinline__ void control_update(Ctl* ctl, const CtlConsts& k) {
  if (ctl->done) { ctl->accepted = 0; return; }
  ctl->attempts++;
  double tau1 = bits_to_tau(ctl->tau_bits[0]);
  double tau2 = bits_to_tau(ctl->tau_bits[1]);
  double tau = tau1 < tau2 ? tau1 : tau2;
  ctl->tau_last = tau;
  const double dt_use = ctl->dt_use;
  if (ctl->status & (kDevNonFinite | kDevCG | kDevTimeout)) {
    ctl->accepted = 0;
    ctl->done = 1;
    return;
  }
  if (ctl->status & kDevTangled) {
    tau = 0.0;
    ctl->status &= ~kDevTangled;
  }
  if (ctl->fixed) {
    ctl->accepted = 1;
    ctl->steps++;
    ctl->t = ctl->t + dt_use;
  } else if (dt_use >= tau) {
    ctl->accepted = 0;
    ctl->rejects++;
    ctl->dt = k.beta1 * dt_use;
    if (ctl->dt < ctl->dt_min) {
      ctl->status |= kDevDtMin;
      ctl->done = 1;
    }
  } else {
    ctl->accepted = 1;
    ctl->steps++;
    if (ctl->dt_log != nullptr && ctl->steps <= ctl->dt_log_cap) ctl->dt_log[ctl->steps - 1] = dt_use;
    ctl->t = ctl->last ? ctl->t_final : ctl->t + dt_use;
    ctl->dt = (dt_use <= k.gamma_dt * tau) ? k.beta2 * dt_use : dt_use;
    if (ctl->last || ctl->steps >= ctl->max_steps) ctl->done = 1;
  }
  if (!ctl->done && !ctl->fixed) {
    double d = ctl->dt;
    ctl->last = 0;
    if (ctl->t + d >= ctl->t_final) {
      d = ctl->t_final - ctl->t;
      ctl->last = 1;
    }
    ctl->dt_use = d;
  }
  ctl->tau_bits[0] = kInfBits;
  ctl->tau_bits[1] = kInfBits;
}

// Start of a run: counters, limits and the first dt_use.  When no step size
// is known yet (dt <= 0) the first one is the estimate of the initial state
// (est_bits, ordered bits).  A fixed-dt replay accepts every attempt.
__device__ __forceinline__ void control_begin(Ctl* ctl, double t_final, long long max_steps,
                                              double dt_min, int fixed, double dt_fixed,
                                              double* dt_log, long long dt_log_cap,
                                              const unsigned long long* est_bits) {
  ctl->t_final = t_final;
  ctl->max_steps = max_steps;
  ctl->dt_min = dt_min;
  ctl->steps = 0;
  ctl->rejects = 0;
  ctl->attempts = 0;
  ctl->cg_iters = 0;
  ctl->done = 0;
  ctl->accepted = 0;
  ctl->status = 0;
  ctl->fixed = fixed;
  ctl->dt_log = dt_log;
  ctl->dt_log_cap = dt_log_cap;
  ctl->tau_bits[0] = kInfBits;
  ctl->tau_bits[1] = kInfBits;
  if (fixed) {
    ctl->dt_use = dt_fixed;
    ctl->last = 0;
    return;
  }
  if (!(ctl->dt > 0.0)) ctl->dt = bits_to_tau(*est_bits);
  double d = ctl->dt;
  ctl->last = 0;
  if (ctl->t + d >= t_final) {
    d = t_final - ctl->t;
    ctl->last = 1;
  }
  ctl->dt_use = d;
  if (ctl->t >= t_final) ctl->done = 1;
}

}  // namespace lagh
