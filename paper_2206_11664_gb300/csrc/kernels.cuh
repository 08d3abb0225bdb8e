// Launch interfaces of the state-vector kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "sd_internal.h"

namespace sd {

// Device copy of a pass schedule.
struct DevSchedule {
    int K = 0, c = 0;
    int64_t n_passes = 0;
    DevPass *passes = nullptr;
    DevRound *rounds = nullptr;
    DevOp *ops = nullptr;
    DevPerm *perms = nullptr;
    DevDiag *diags = nullptr;
    DevPhase *phases = nullptr;
    uint64_t *term_mo = nullptr;
    DevSlot *slots = nullptr;
    int64_t *term_q = nullptr;
    uint64_t *mask_pool = nullptr;
    uint64_t *cst_mo = nullptr;
    int64_t *cst_q = nullptr;
    const double2 *tw = nullptr;       // per-device constant tables (not owned)
    const longlong2 *fxt = nullptr;
    std::vector<DevPass> host_passes;  // for launch-side decisions
};

// Device copy of a flat circuit for the on-chip path (whole state in smem).
struct DevFlatOp {
    int32_t kind, q, q2, idx;
};
struct DevDiagFlat {
    int64_t begin, count;   // into masks/q pools
};
struct DevCircuit {
    int64_t n_ops = 0;
    DevFlatOp *ops = nullptr;
    DevDiagFlat *diags = nullptr;
    uint64_t *dmasks = nullptr;
    int64_t *dq = nullptr;
    uint64_t *phase_sp = nullptr, *phase_sm = nullptr;   // per phase layer
    uint64_t *phase_up = nullptr;                         // n per phase layer
};

// One instance of a level-synchronous batch: at level L it runs the L-th pass
// of its sequence head (npass[0] passes), core x reps_core, tail (npass[2]),
// on blocks [cta_begin, cta_begin + cta_count) of the launch.
struct BatchInstance {
    void *psi;
    int n;
    int cta_begin, cta_count;
    int npass[3];
    int64_t reps_core;
    int64_t levels;
    KParams kp[3];
};

// Launch level `level` of a batch whose instances all use tile size K;
// cta_inst maps each block to its instance; smem = the largest pass need.
cudaError_t launch_tile_pass_batch(bool dbl, int K, const BatchInstance *d_inst, const uint16_t *d_cta_inst,
                                   int blocks, size_t smem, int64_t level, cudaStream_t st);

int tile_pass_batch_occupancy(bool dbl, int K, size_t smem);

// Dynamic shared memory of a tile pass and its limit.

cudaError_t launch_tile_pass(bool dbl, void *psi, int n, const DevSchedule &S, int pass,
                             int num_sms, cudaStream_t st);

// Whole evolution on chip (n <= onchip_max_qubits): `reps` repetitions of
// the circuit; if obs_terms > 0, after every repetition writes
// sum_k oc[k] <psi|Z^{oz[k]}|psi> to trace[rep].
cudaError_t launch_onchip(bool dbl, void *psi, int n, const DevCircuit &C, int64_t reps,
                          const uint64_t *d_oz, const double *d_oc, int obs_terms,
                          double *d_trace, cudaStream_t st);
int onchip_max_qubits(bool dbl);

cudaError_t launch_pauli_rotation(bool dbl, void *psi, int n, uint64_t x, uint64_t z,
                                  double c, double s, int num_sms, cudaStream_t st);

// partial[b] for b < blocks: block sums of sum_k oc_k Re <psi|P_k|psi> over
// the given terms (all with the same x mask if x != 0; any z masks).
cudaError_t launch_expect_diag(bool dbl, const void *psi, int n, const uint64_t *d_oz,
                               const double *d_oc, int terms, double *partial, int blocks,
                               cudaStream_t st);
cudaError_t launch_expect_pauli(bool dbl, const void *psi, int n, uint64_t x, uint64_t z,
                                double coef, double *partial, int blocks, cudaStream_t st);
// out[0] (+)= sum of partial[0..count) in fixed order.
cudaError_t launch_copy16(const void *src, void *dst, size_t bytes, int num_sms, cudaStream_t st);
cudaError_t launch_reduce(const double *partial, int64_t count, double *out, int accumulate,
                          cudaStream_t st);

// lam <- sum_k oc_k P_k phi  (lam zeroed first).
cudaError_t launch_apply_observable(bool dbl, const void *phi, void *lam, int n,
                                    const uint64_t *d_ox, const uint64_t *d_oz, const double *d_oc,
                                    int terms, cudaStream_t st);

// Gradient step at a group's diagonal point: chi, mu are C_g phi, C_g lambda.
// Adds to partial[block][j] the sums sum_x Im(conj(mu_x) chi_x) (-1)^{|x & m_j|}
// for the group's terms (classes by the low 4 index bits), then applies the
// inverse group exponential to chi and mu.
struct DevGrad {
    int32_t off[17];
    int32_t m;             // number of terms in the group
    int64_t base;          // into masks_f / q / term_id pools
};
cudaError_t launch_grad_diag(bool dbl, void *chi, void *mu, int n, const DevGrad &g,
                             const uint64_t *masks_f, const int64_t *qinv,
                             const longlong2 *fxt, double *partial, int blocks,
                             cudaStream_t st);
int grad_blocks(int n, int num_sms);

cudaError_t launch_copy(void *dst, const void *src, size_t bytes, cudaStream_t st);

}  // namespace sd

namespace sd {
// gacc[term_id[j]] += factor[j] * sum_b partial[b * m + j]  for j < m.
cudaError_t launch_grad_finalize(const double *partial, int blocks, int m, const int32_t *term_id,
                                 const double *factor, double *gacc, cudaStream_t st);
}  // namespace sd
