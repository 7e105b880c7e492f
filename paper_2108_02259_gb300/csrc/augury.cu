// apic_augury_steps: augury dynamics (Sec. 2.2, eq. apic_accel with
// eq. Newmark read as velocity Verlet) on the device, with a linear-spring
// foreground and uniform gravity.  Each step runs the kernels of kernels.cu
// around two calls of this library's own entry points: apic_node_normals
// (Sec. 2.3 normals at the new positions) and apic_contact_step (the
// preferred velocity V_hat of the predicted V_bar).
#include <cstring>

#include "pipeline.cuh"

using namespace apic;

namespace {

template <class U>
apic_status take(apic_ctx* c, int slot, size_t count, U** out) {
  void* p = nullptr;
  P_TRY(ctx_take(c, slot, count * sizeof(U), &p));
  *out = static_cast<U*>(p);
  return APIC_OK;
}

template <class T>
apic_status run_augury(apic_ctx* c, const apic_augury_args* a, int32_t n_steps, cudaStream_t s,
                       apic_augury_stats* stats) {
  const int64_t n = a->n;
  double* f;
  T *am, *vbar, *vhat, *Chat, *nrm;
  double* out;  // [0..2] energies, [3] spring index error flag (as int), [4..9] P, L
  P_TRY(take(c, kSlotAugF, 3 * n, &f));
  P_TRY(take(c, kSlotAugAm, 3 * n, &am));
  P_TRY(take(c, kSlotAugVbar, 3 * n, &vbar));
  P_TRY(take(c, kSlotAugVhat, 3 * n, &vhat));
  P_TRY(take(c, kSlotAugChat, 9 * n, &Chat));
  P_TRY(take(c, kSlotAugNrm, 3 * n, &nrm));
  P_TRY(take(c, kSlotAugOut, 16, &out));
  int* err = reinterpret_cast<int*>(out + 3);
  P_CUDA(cudaMemsetAsync(out, 0, 16 * sizeof(double), s));
  if (a->n_tri == 0) P_CUDA(cudaMemsetAsync(nrm, 0, 3 * n * sizeof(T), s));

  T* v = static_cast<T*>(a->v);
  T* C = static_cast<T*>(a->C);
  T* av = static_cast<T*>(a->av);
  T* aC = static_cast<T*>(a->aC);
  const T* m = static_cast<const T*>(a->m);
  const double dt = a->dt, tau = a->tau;

  apic_step_args sa{};
  sa.n = n;
  sa.n_bodies = a->n_bodies;
  sa.n_iter = a->n_iter;
  sa.body = a->body;
  sa.x = a->x;
  sa.v = vbar;
  sa.C = C;  // C_bar = C (no mechanical rate on the affine mode)
  sa.m = m;
  sa.nrm = nrm;
  sa.v_out = vhat;
  sa.C_out = Chat;
  sa.h = a->h;
  sa.mu = a->mu;
  sa.mu_pair = a->mu_pair;
  sa.flags = a->flags & (APIC_FP64 | APIC_VARIANT_PIC | APIC_VARIANT_SEP23);

  // A = {a, 0} + (V_hat - V_bar) / tau with V_bar = V + c_bar {a, 0}; then V += half_dt A
  auto accelerate = [&](double c_bar, double half_dt) -> apic_status {
    if (a->n_tri > 0)
      P_TRY(apic_node_normals(c, n, a->x, a->n_tri, a->tri, nrm, a->flags & APIC_FP64, s));
    P_CUDA(cudaMemsetAsync(f, 0, 3 * n * sizeof(double), s));
    P_CUDA(launch_aug_springs(a->n_springs, a->springs, a->rest, a->stiffness, a->x, n, f, err, s));
    P_CUDA(launch_aug_predict<T>(n, f, m, a->gravity, v, am, vbar, (T)c_bar, s));
    P_TRY(apic_contact_step(c, &sa, s, nullptr));
    P_CUDA(launch_aug_finish<T>(n, am, vbar, vhat, Chat, a->fixed, (T)(1.0 / tau), (T)half_dt, v, C, av, aC, s));
    return APIC_OK;
  };
  if (a->flags & APIC_AUGURY_INIT) P_TRY(accelerate(tau, 0.0));
  for (int32_t step = 0; step < n_steps; ++step) {
    P_CUDA(launch_aug_kick_drift<T>(n, a->x, v, C, av, aC, a->fixed, (T)(0.5 * dt), dt, s));
    P_TRY(accelerate(0.5 * dt + tau, 0.5 * dt));
  }
  if (stats) {
    P_CUDA(launch_aug_energy<T>(n, a->x, v, m, a->gravity, a->n_springs, a->springs, a->rest, a->stiffness, out, s));
    P_CUDA(launch_momentum<T>(n, a->x, v, C, m, a->h, out + 4, s));
  }
  double h_out[16];
  P_CUDA(cudaMemcpyAsync(h_out, out, sizeof(h_out), cudaMemcpyDeviceToHost, s));
  P_CUDA(cudaStreamSynchronize(s));
  int e = 0;
  std::memcpy(&e, &h_out[3], sizeof(int));
  if (e) return pfail(APIC_ERR_INVALID_ARG, "a spring index is outside [0, %lld)", (long long)n);
  if (stats) {
    stats->kinetic = h_out[0];
    stats->springs = h_out[1];
    stats->gravity = h_out[2];
    for (int k = 0; k < 3; ++k) {
      stats->P[k] = h_out[4 + k];
      stats->L[k] = h_out[7 + k];
    }
  }
  return APIC_OK;
}

}  // namespace

extern "C" apic_status apic_augury_steps(apic_ctx* c, const apic_augury_args* a, int32_t n_steps, void* stream,
                                         apic_augury_stats* stats) {
  if (!c || !a) return pfail(APIC_ERR_INVALID_ARG, "NULL argument");
  if (a->n <= 0) return pfail(APIC_ERR_INVALID_ARG, "n = %lld must be > 0", (long long)a->n);
  if (n_steps < 0) return pfail(APIC_ERR_INVALID_ARG, "n_steps = %d < 0", n_steps);
  if (!(a->dt > 0.0) || !(a->tau > 0.0))
    return pfail(APIC_ERR_INVALID_ARG, "dt = %g and tau = %g must be > 0", a->dt, a->tau);
  if (a->n_springs < 0 || a->n_tri < 0) return pfail(APIC_ERR_INVALID_ARG, "negative spring or triangle count");
  if (!a->x || !a->v || !a->C || !a->av || !a->aC || !a->m || !a->body ||
      (a->n_springs > 0 && (!a->springs || !a->rest || !a->stiffness)) || (a->n_tri > 0 && !a->tri))
    return pfail(APIC_ERR_INVALID_ARG, "a required array pointer is NULL");
  const uint32_t allowed = APIC_FP64 | APIC_VARIANT_PIC | APIC_VARIANT_SEP23 | APIC_AUGURY_INIT;
  if (a->flags & ~allowed)
    return pfail(APIC_ERR_INVALID_ARG, "flag bits 0x%x not accepted here (device pointers only)", a->flags & ~allowed);
  if (stats) std::memset(stats, 0, sizeof(*stats));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return (a->flags & APIC_FP64) ? run_augury<double>(c, a, n_steps, s, stats)
                                : run_augury<float>(c, a, n_steps, s, stats);
}
