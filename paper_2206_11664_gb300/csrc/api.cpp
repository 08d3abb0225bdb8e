// C ABI (include/sd.h): contexts, planning, device programs and the drivers
// of evolution, expectation and gradient.  All state-vector work is done by
// the kernels in kernels.cu; this file only plans, schedules, uploads and
// launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <list>
#include <memory>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/sd.h"
#include "jit.h"
#include "kernels.cuh"
#include "sd_internal.h"

using namespace sd;

namespace {

thread_local std::string g_last_error;

// Device program of one circuit: either a pass schedule (tile path) or a
// flat op list (on-chip path).
struct Program {
    bool onchip = false;
    DevSchedule sched;
    JitProgram jit;           // run-time specialised passes, if built
    DevCircuit circ;
    std::vector<void *> allocs;
    int64_t passes = 0, rounds = 0, diag_passes = 0;
    // the pass launches of one repetition, as CUDA graphs, for up to 4 states
    std::vector<std::pair<void *, cudaGraphExec_t>> graphs;
};

struct GradGroup {   // per (group, fraction): class-sorted terms for the adjoint kernel
    DevGrad g{};
    uint64_t *masks_f = nullptr;
    int64_t *qinv = nullptr;
    int32_t *term_id = nullptr;
    double *factor = nullptr;
};

void free_program(Program &p) {
    for (auto &g : p.graphs) cudaGraphExecDestroy(g.second);
    p.graphs.clear();
    for (void *a : p.allocs) cudaFree(a);
    p.allocs.clear();
}

}  // namespace

namespace {
void batch_purge(const sd_ctx *ctx);
}

struct sd_ctx {
    int n = 0;
    int64_t m = 0;
    std::vector<uint64_t> x, z;
    std::vector<double> c;
    bool planned = false;
    Plan plan;
    int tile_bits_opt = 0;
    int tuned_k[2] = {0, 0};   // tile size chosen by sd_autotune (complex64, complex128)
    int jit_opt = 0;
    int layout_opt = 0;        // sd_plan_opts.layout
    int tuned_layout = 0;      // complex64 layout chosen by sd_autotune_shape (1 paired, -1 plain)
    int prefetch_opt = 0;      // sd_plan_opts.prefetch
    int tuned_prefetch[2] = {0, 0};   // prefetch buffers chosen by sd_autotune_shape (per dtype)
    std::string jit_note;    // why the last program did not use run-time specialisation
    // plan view storage
    std::vector<int64_t> v_goff, v_gterms, v_gateoff;
    std::vector<uint64_t> v_masks, v_cols, v_icols;
    std::vector<uint8_t> v_signs;
    std::vector<int32_t> v_gates;
    std::string err;
    // device side
    int num_sms = 0;
    std::map<std::tuple<int, int, int, double>, std::unique_ptr<Program>> programs;
    std::map<std::tuple<int, int, int>, std::unique_ptr<Program>> cliff_programs;   // (dtype, group, fwd)
    std::map<std::tuple<int, int, int>, std::unique_ptr<Program>> transition_programs;   // (dtype, from, to)
    std::map<std::pair<int, double>, GradGroup> grad_groups;
    std::vector<void *> grad_allocs;
    double *d_partial = nullptr;
    size_t partial_cap = 0;
    double *d_scalar = nullptr;
    uint64_t *d_obs = nullptr;   // ox | oz | oc staging
    size_t obs_cap = 0;
    void *d_work[2] = {nullptr, nullptr};
    size_t work_bytes = 0;
    double *d_gacc = nullptr;
    double grad_dt = 0.0;
    cudaStream_t graph_stream = nullptr;   // private stream for capturing pass graphs

    ~sd_ctx() {
        batch_purge(this);
        for (auto &kv : programs) free_program(*kv.second);
        for (auto &kv : cliff_programs) free_program(*kv.second);
        for (auto &kv : transition_programs) free_program(*kv.second);
        for (void *a : grad_allocs) cudaFree(a);
        cudaFree(d_partial);
        cudaFree(d_scalar);
        cudaFree(d_obs);
        cudaFree(d_work[0]);
        cudaFree(d_work[1]);
        cudaFree(d_gacc);
        if (graph_stream) cudaStreamDestroy(graph_stream);
    }
};

namespace {

sd_status fail(sd_ctx *ctx, sd_status s, const std::string &msg) {
    g_last_error = msg;
    if (ctx) ctx->err = msg;
    return s;
}

#define CK(call)                                                                         \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(ctx, SD_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <typename T>
cudaError_t upload(std::vector<void *> &allocs, T *&dst, const std::vector<T> &src) {
    size_t bytes = sizeof(T) * std::max<size_t>(src.size(), 1);
    cudaError_t e = cudaMalloc((void **)&dst, bytes);
    if (e != cudaSuccess) return e;
    allocs.push_back(dst);
    if (!src.empty()) e = cudaMemcpy(dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice);
    return e;
}

sd_status ensure_device(sd_ctx *ctx) {
    if (ctx->num_sms) return SD_OK;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, dev));
    return SD_OK;
}

// Constant rotation tables, one copy per device for the life of the process,
// computed on the host in long double: e^{2 pi i k/256} in FP64, and the
// Q1.62 tables of the fixed-point passes (e^{2 pi i k/256}, e^{2 pi i k/65536}).
struct DevTables {
    double2 *tw = nullptr;
    longlong2 *fxt = nullptr;
};
std::mutex g_tab_mu;
std::map<int, DevTables> g_tabs;

sd_status device_tables(sd_ctx *ctx, DevTables &out) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_tab_mu);
    auto it = g_tabs.find(dev);
    if (it != g_tabs.end()) {
        out = it->second;
        return SD_OK;
    }
    const long double pi = 3.141592653589793238462643383279502884L;
    std::vector<double2> tw(768);
    std::vector<longlong2> fxt(512);
    for (int k = 0; k < 512; k++) {
        const long double a = 2.0L * pi * k / 512.0L;
        tw[256 + k] = make_double2((double)cosl(a), (double)sinl(a));
    }
    for (int k = 0; k < 256; k++) {
        const long double a = 2.0L * pi * k / 256.0L, b = 2.0L * pi * k / 65536.0L;
        tw[k] = make_double2((double)cosl(a), (double)sinl(a));
        fxt[k] = make_longlong2(llroundl(ldexpl(cosl(a), 62)), llroundl(ldexpl(sinl(a), 62)));
        fxt[256 + k] = make_longlong2(llroundl(ldexpl(cosl(b), 62)), llroundl(ldexpl(sinl(b), 62)));
    }
    DevTables t;
    CK(cudaMalloc((void **)&t.tw, sizeof(double2) * tw.size()));
    CK(cudaMalloc((void **)&t.fxt, sizeof(longlong2) * fxt.size()));
    CK(cudaMemcpy(t.tw, tw.data(), sizeof(double2) * tw.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(t.fxt, fxt.data(), sizeof(longlong2) * fxt.size(), cudaMemcpyHostToDevice));
    g_tabs[dev] = t;
    out = t;
    return SD_OK;
}

int default_tile_bits(const sd_ctx *ctx, bool dbl) {
    int K = ctx->tile_bits_opt > 0 ? ctx->tile_bits_opt
            : ctx->tuned_k[dbl ? 1 : 0] > 0 ? ctx->tuned_k[dbl ? 1 : 0] : (dbl ? 12 : 13);
    return std::min(K, ctx->n);
}

bool use_onchip(const sd_ctx *ctx, bool dbl) { return ctx->n <= onchip_max_qubits(dbl); }

// Most tile passes of one program compiled at run time (per-pass kernels).
constexpr int64_t kJitMaxPasses = 512;
// Steps (first order) or cores (second order) merged into one block program.
constexpr int kBlockSteps = 4;

// Appends circuit b to circuit a (table indices of b's diagonal ops rebased).
void append_circuit(Circuit &a, const Circuit &b) {
    const int32_t np = (int32_t)a.phases.size(), nd = (int32_t)a.diags.size();
    for (FlatOp op : b.ops) {
        if (op.kind == OK_PHASE) op.idx += np;
        else if (op.kind == OK_DIAG) op.idx += nd;
        a.ops.push_back(op);
    }
    a.phases.insert(a.phases.end(), b.phases.begin(), b.phases.end());
    a.diags.insert(a.diags.end(), b.diags.begin(), b.diags.end());
}

// Pass schedule of a canonicalised circuit on the tile path: the default
// tile size, or smaller tiles when a pass's staged terms do not fit beside
// the tile in shared memory.
// Circuits up to this many ops are scheduled twice, with and without
// deferring single-gate last rounds (schedule_circuit), and the schedule with
// fewer passes, then fewer rounds, is kept.
constexpr size_t kTailTrialOps = 20000;

sd_status schedule_for(sd_ctx *ctx, const Circuit &circ, bool dbl, Schedule &S, bool pin0 = false) {
    int K = default_tile_bits(ctx, dbl);
    const int c = dbl ? 3 : 4;
    auto need_of = [&](const Schedule &X) {
        size_t need = 0;
        for (auto &p : X.passes) need = std::max(need, pass_smem_bytes(p, dbl ? 16 : 8, K));
        return need;
    };
    for (;;) {
        std::string e = schedule_circuit(circ, ctx->n, K, c, S, pin0);
        if (!e.empty()) return fail(ctx, SD_EINTERNAL, "scheduler: " + e);
        if (need_of(S) <= kTileSmemLimit) {
            if (circ.ops.size() <= kTailTrialOps) {
                Schedule T;
                if (schedule_circuit(circ, ctx->n, K, c, T, pin0, true).empty() && need_of(T) <= kTileSmemLimit &&
                    (T.passes.size() < S.passes.size() ||
                     (T.passes.size() == S.passes.size() && T.rounds.size() < S.rounds.size())))
                    S = std::move(T);
            }
            return SD_OK;
        }
        if (K <= kRegBits + kLaneBits)
            return fail(ctx, SD_EINVAL, "a commuting group has too many terms for one tile pass");
        K--;   // smaller tiles leave room to stage the group's terms
    }
}

// Whether a program of `passes` tile passes is compiled at run time: always
// with jit = 1 (or SD_JIT=1), never with jit = -1 (or SD_JIT=0), else for
// states of 20+ qubits and at most kJitMaxPasses passes.  The one-shot
// program that opens a second-order evolution (group 1's half step,
// allow_jit = false) is not worth a compilation unless it is forced.  The
// closing program is the core with group 1's last exponential halved: the
// same passes with other angles, whose generated source (angles are kernel
// arguments) is the core's, so that its kernels come from the core's cache.
bool jit_wanted(const sd_ctx *ctx, bool allow_jit, int64_t passes) {
    int mode = ctx->jit_opt;
    if (const char *e = getenv("SD_JIT")) mode = atoi(e) > 0 ? 1 : (e[0] == '0' ? -1 : mode);
    if (passes <= 0) return false;
    return mode > 0 || (mode == 0 && allow_jit && ctx->n >= 20 && passes <= kJitMaxPasses);
}

// The two-buffer prefetch form the shape autotuner tries for a dtype: for
// complex64 two buffers in the passes without a group exponential only (the
// light passes wait on their loads; the exponential passes gain nothing), for
// complex128 two in every pass.
int two_buffer_form(bool dbl) { return dbl ? 2 : 3; }
// Prefetch depth of the run-time passes (sd_plan_opts.prefetch): sd_plan's
// choice, else the tuned one, else one buffer for complex64 and two for
// complex128.
int prefetch_buffers(const sd_ctx *ctx, bool dbl) {
    if (ctx->prefetch_opt > 0) return ctx->prefetch_opt;
    const int t = ctx->tuned_prefetch[dbl ? 1 : 0];
    return t > 0 ? t : (dbl ? 2 : 1);
}

// With the paired layout, complex64 programs that will probably be compiled
// at run time are scheduled with tile position 0 pinned to register slot 0,
// which the paired pass code needs (the interpreter runs such schedules as
// well, should the compilation not happen).
bool pin0_wanted(const sd_ctx *ctx, bool dbl, bool allow_jit) {
    if (dbl) return false;
    const int layout = ctx->layout_opt != 0 ? ctx->layout_opt : ctx->tuned_layout;
    return layout > 0 && jit_wanted(ctx, allow_jit, 1);
}

// Build and upload a program for a circuit.
sd_status build_program(sd_ctx *ctx, const Circuit &circ_in, bool dbl, Program &P,
                        bool allow_jit = true) {
    P.onchip = use_onchip(ctx, dbl);
    Circuit circ = circ_in;
    canonicalize_1q(circ, ctx->n);
    const int n = ctx->n;
    if (P.onchip) {
        std::vector<DevFlatOp> ops;
        for (auto &o : circ.ops) ops.push_back(DevFlatOp{o.kind, o.q, o.q2, o.idx});
        std::vector<DevDiagFlat> dg;
        std::vector<uint64_t> dm;
        std::vector<int64_t> dq;
        for (auto &d : circ.diags) {
            dg.push_back(DevDiagFlat{(int64_t)dm.size(), (int64_t)d.masks.size()});
            dm.insert(dm.end(), d.masks.begin(), d.masks.end());
            dq.insert(dq.end(), d.q.begin(), d.q.end());
        }
        std::vector<uint64_t> sp, smk, up;
        for (auto &L : circ.phases) {
            sp.push_back(L.sp);
            smk.push_back(L.sm);
            up.insert(up.end(), L.up.begin(), L.up.end());
        }
        DevCircuit &C = P.circ;
        C.n_ops = (int64_t)ops.size();
        CK(upload(P.allocs, C.ops, ops));
        CK(upload(P.allocs, C.diags, dg));
        CK(upload(P.allocs, C.dmasks, dm));
        CK(upload(P.allocs, C.dq, dq));
        CK(upload(P.allocs, C.phase_sp, sp));
        CK(upload(P.allocs, C.phase_sm, smk));
        CK(upload(P.allocs, C.phase_up, up));
        P.passes = 0;
        return SD_OK;
    }
    Schedule S;
    sd_status ss = schedule_for(ctx, circ, dbl, S, pin0_wanted(ctx, dbl, allow_jit));
    if (ss != SD_OK) return ss;
    S.prefetch = prefetch_buffers(ctx, dbl);
    DevSchedule &D = P.sched;
    DevTables tabs;
    if ((ss = device_tables(ctx, tabs)) != SD_OK) return ss;
    D.tw = tabs.tw;
    D.fxt = tabs.fxt;
    D.K = S.K;
    D.c = S.c;
    D.n_passes = (int64_t)S.passes.size();
    D.host_passes = S.passes;
    CK(upload(P.allocs, D.passes, S.passes));
    CK(upload(P.allocs, D.rounds, S.rounds));
    CK(upload(P.allocs, D.ops, S.ops));
    CK(upload(P.allocs, D.perms, S.perms));
    CK(upload(P.allocs, D.diags, S.diags));
    CK(upload(P.allocs, D.phases, S.phases));
    CK(upload(P.allocs, D.term_mo, S.term_mo));
    CK(upload(P.allocs, D.slots, S.slots));
    CK(upload(P.allocs, D.term_q, S.term_q));
    CK(upload(P.allocs, D.mask_pool, S.mask_pool));
    CK(upload(P.allocs, D.cst_mo, S.cst_mo));
    CK(upload(P.allocs, D.cst_q, S.cst_q));
    P.passes = (int64_t)S.passes.size();
    P.rounds = (int64_t)S.rounds.size();
    P.diag_passes = S.diag_passes;
    if (jit_wanted(ctx, allow_jit, P.passes)) {
        std::string why = jit_build(S, n, dbl, P.jit);
        if (!why.empty()) {
            P.jit = JitProgram{};
            ctx->jit_note = why;
        }
    }
    return SD_OK;
}

// Group order and fractions of one Trotter step.
std::vector<std::pair<int, double>> step_sequence(int G, int order) {
    std::vector<std::pair<int, double>> s;
    if (order == 1 || G == 1) {
        for (int g = 0; g < G; g++) s.push_back({g, 1.0});
        return s;
    }
    for (int g = 0; g < G - 1; g++) s.push_back({g, 0.5});
    s.push_back({G - 1, 1.0});
    for (int g = G - 2; g >= 0; g--) s.push_back({g, 0.5});
    return s;
}

// Segments of an evolution: kind 0 = one unmerged step, 1 = head, 2 = core, 3 = tail
// (second order with half steps of group 0 merged across steps), 4 = block:
// kBlockSteps (or fewer, see block_steps) repetitions of the step (first
// order) or of the core (second order) in one program, so that the schedule
// runs the last Clifford layer of one step in the passes of the next step's
// first group exponential instead of in passes of its own.
Circuit segment_circuit(const sd_ctx *ctx, int order, int kind, double dt, int reps = 1) {
    Circuit c;
    const int G = (int)ctx->plan.groups.size();
    if (kind == 4) {
        const int base = (order == 1 || G == 1) ? 0 : 2;
        for (int r = 0; r < reps; r++) {
            Circuit one = segment_circuit(ctx, order, base, dt);
            append_circuit(c, one);
        }
        return c;
    }
    auto add = [&](int g, double f) { append_group_step(ctx->plan, g, f, dt, ctx->c, c); };
    if (kind == 0 || order == 1 || G == 1) {
        for (auto &p : step_sequence(G, order)) add(p.first, p.second);
        return c;
    }
    if (kind == 1) {
        add(0, 0.5);
        return c;
    }
    for (int g = 1; g < G - 1; g++) add(g, 0.5);
    add(G - 1, 1.0);
    for (int g = G - 2; g >= 1; g--) add(g, 0.5);
    add(0, kind == 2 ? 1.0 : 0.5);
    return c;
}

sd_status get_program(sd_ctx *ctx, bool dbl, int order, int kind, double dt, Program *&out, int reps = 1) {
    auto key = std::make_tuple((int)dbl, order, kind * 64 + reps, dt);
    auto it = ctx->programs.find(key);
    if (it != ctx->programs.end()) {
        out = it->second.get();
        return SD_OK;
    }
    // keep the cache small: programs for other dt values are dropped
    for (auto i = ctx->programs.begin(); i != ctx->programs.end();) {
        if (std::get<3>(i->first) != dt) {
            batch_purge(ctx);
            free_program(*i->second);
            i = ctx->programs.erase(i);
        } else {
            ++i;
        }
    }
    auto P = std::make_unique<Program>();
    Circuit c = segment_circuit(ctx, order, kind, dt, reps);
    sd_status s = build_program(ctx, c, dbl, *P, kind != 1);
    if (s != SD_OK) {
        free_program(*P);
        return s;
    }
    out = P.get();
    ctx->programs[key] = std::move(P);
    return SD_OK;
}

// States up to this size run their pass sequences as CUDA graphs.
constexpr size_t kGraphMaxStateBytes = (size_t)256 << 20;

// The pass launches of one repetition of a tile-path program.
sd_status launch_passes(sd_ctx *ctx, bool dbl, Program &P, void *psi, cudaStream_t st) {
    if (P.jit.ok()) {
        const KParams kp{P.sched.passes, P.sched.rounds, P.sched.ops, P.sched.perms, P.sched.diags,
                         P.sched.phases, P.sched.term_mo, P.sched.slots, P.sched.term_q,
                         P.sched.mask_pool, P.sched.cst_mo, P.sched.cst_q, P.sched.c,
                         P.sched.tw, P.sched.fxt};
        for (int64_t p = 0; p < P.sched.n_passes; p++)
            CK(jit_launch(P.jit, (int)p, psi, kp, ctx->n, ctx->num_sms, st));
        return SD_OK;
    }
    for (int64_t p = 0; p < P.sched.n_passes; p++)
        CK(launch_tile_pass(dbl, psi, ctx->n, P.sched, (int)p, ctx->num_sms, st));
    return SD_OK;
}

sd_status run_program(sd_ctx *ctx, bool dbl, Program &P, void *psi, int64_t reps, cudaStream_t st,
                      const uint64_t *d_oz = nullptr, const double *d_oc = nullptr, int nobs = 0,
                      double *d_trace = nullptr) {
    if (reps <= 0) return SD_OK;
    if (P.onchip) {
        if (P.circ.n_ops == 0 && nobs == 0) return SD_OK;
        CK(launch_onchip(dbl, psi, ctx->n, P.circ, reps, d_oz, d_oc, nobs, d_trace, st));
        return SD_OK;
    }
    // Small states make the passes launch-bound: their launches are then
    // captured once into a CUDA graph (per program and state) and replayed.
    const size_t state_bytes = ((size_t)1 << ctx->n) * (dbl ? 16 : 8);
    bool use_graph = state_bytes <= kGraphMaxStateBytes && P.sched.n_passes >= 8;
    if (use_graph) {
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
            cudaGetLastError();
            use_graph = false;   // the caller is capturing: launch into its graph directly
        }
    }
    cudaGraphExec_t graph = nullptr;
    if (use_graph)
        for (auto &g : P.graphs)
            if (g.first == psi) graph = g.second;
    if (use_graph && !graph) {
        if (!ctx->graph_stream) CK(cudaStreamCreateWithFlags(&ctx->graph_stream, cudaStreamNonBlocking));
        if (P.graphs.size() >= 4) {
            cudaGraphExecDestroy(P.graphs.front().second);
            P.graphs.erase(P.graphs.begin());
        }
        CK(cudaStreamBeginCapture(ctx->graph_stream, cudaStreamCaptureModeThreadLocal));
        sd_status s = launch_passes(ctx, dbl, P, psi, ctx->graph_stream);
        cudaGraph_t g = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(ctx->graph_stream, &g);
        if (s != SD_OK) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        if (ee != cudaSuccess) return fail(ctx, SD_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ee));
        const cudaError_t ie = cudaGraphInstantiate(&graph, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) return fail(ctx, SD_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ie));
        P.graphs.push_back({psi, graph});
    }
    for (int64_t r = 0; r < reps; r++) {
        if (use_graph) {
            CK(cudaGraphLaunch(graph, st));
        } else {
            sd_status s = launch_passes(ctx, dbl, P, psi, st);
            if (s != SD_OK) return s;
        }
    }
    return SD_OK;
}

sd_status check_state_args(sd_ctx *ctx, const void *state, sd_dtype dtype, int order) {
    if (!ctx) return fail(nullptr, SD_EINVAL, "null context");
    if (!ctx->planned) return fail(ctx, SD_ENOPLAN, "sd_plan has not been called");
    if (!state) return fail(ctx, SD_EINVAL, "null state pointer");
    if (dtype != SD_C64 && dtype != SD_C128) return fail(ctx, SD_EINVAL, "dtype must be SD_C64 or SD_C128");
    if (order != 1 && order != 2) return fail(ctx, SD_EINVAL, "order must be 1 or 2");
    // the passes move 16 bytes per copy (two complex64 or one complex128 amplitude)
    if ((uintptr_t)state % 16 != 0) return fail(ctx, SD_EINVAL, "state must be 16-byte aligned");
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, state) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return fail(ctx, SD_EINVAL, "state must be a device pointer");
    }
    return ensure_device(ctx);
}

// Repetitions of a segment of `passes` tile passes merged into one block
// program: kBlockSteps, halved until the block stays within the limit of run-time
// compiled passes; 1 (no block) for the on-chip path.
int block_steps(int64_t passes) {
    if (passes <= 0) return 1;
    int M = kBlockSteps;
    while (M > 1 && M * passes > kJitMaxPasses) M /= 2;
    return M;
}

// Runs `count` repetitions of the segment program R: whole blocks of M
// repetitions through the block program, the rest through R itself.
// (launch = false: only build the programs the call would run.)
sd_status run_repeated(sd_ctx *ctx, bool dbl, int order, double dt, Program &R, int64_t count, void *psi,
                       cudaStream_t st, bool launch) {
    const int M = block_steps(R.passes);
    if (M > 1 && count >= M) {
        Program *B = nullptr;
        sd_status s = get_program(ctx, dbl, order, 4, dt, B, M);
        if (s != SD_OK) return s;
        if (launch && (s = run_program(ctx, dbl, *B, psi, count / M, st)) != SD_OK) return s;
        count %= M;
    }
    return launch ? run_program(ctx, dbl, R, psi, count, st) : SD_OK;
}

sd_status evolve_impl(sd_ctx *ctx, void *psi, bool dbl, double dt, int64_t steps, int order,
                      cudaStream_t st, bool launch = true) {
    const int G = (int)ctx->plan.groups.size();
    Program *P = nullptr;
    sd_status s;
    if (order == 1 || G == 1 || steps == 1) {
        if ((s = get_program(ctx, dbl, order, 0, dt, P)) != SD_OK) return s;
        return run_repeated(ctx, dbl, order, dt, *P, steps, psi, st, launch);
    }
    Program *H = nullptr, *C = nullptr, *T = nullptr;
    if ((s = get_program(ctx, dbl, order, 1, dt, H)) != SD_OK) return s;
    if ((s = get_program(ctx, dbl, order, 2, dt, C)) != SD_OK) return s;
    if ((s = get_program(ctx, dbl, order, 3, dt, T)) != SD_OK) return s;
    if (launch && (s = run_program(ctx, dbl, *H, psi, 1, st)) != SD_OK) return s;
    if ((s = run_repeated(ctx, dbl, order, dt, *C, steps - 1, psi, st, launch)) != SD_OK) return s;
    return launch ? run_program(ctx, dbl, *T, psi, 1, st) : SD_OK;
}

// Tile passes of a segment's schedule, host only (0 on the on-chip path).
sd_status segment_passes(sd_ctx *ctx, bool dbl, int order, int kind, int reps, int64_t &out) {
    out = 0;
    if (use_onchip(ctx, dbl)) return SD_OK;
    Circuit c = segment_circuit(ctx, order, kind, 0.01, reps);
    canonicalize_1q(c, ctx->n);
    Schedule S;
    sd_status s = schedule_for(ctx, c, dbl, S, pin0_wanted(ctx, dbl, kind != 1));
    if (s == SD_OK) out = (int64_t)S.passes.size();
    return s;
}

sd_status ensure_partial(sd_ctx *ctx, size_t count) {
    if (count <= ctx->partial_cap) return SD_OK;
    cudaFree(ctx->d_partial);
    ctx->d_partial = nullptr;
    ctx->partial_cap = 0;
    CK(cudaMalloc((void **)&ctx->d_partial, sizeof(double) * count));
    ctx->partial_cap = count;
    if (!ctx->d_scalar) CK(cudaMalloc((void **)&ctx->d_scalar, sizeof(double) * 4));
    return SD_OK;
}

int expect_blocks(const sd_ctx *ctx) {
    int64_t N = (int64_t)1 << ctx->n;
    int64_t b = (N + 255) / 256;
    int64_t cap = (int64_t)ctx->num_sms * 4;
    return (int)std::max<int64_t>(1, std::min(b, cap));
}

// Observable staged on the device: diagonal terms (x = 0) packed for one
// fused pass, the others kept on the host for one pass each.
struct StagedObs {
    int nd = 0;
    const uint64_t *dz = nullptr;
    const double *dc = nullptr;
    std::vector<uint64_t> ox, oz;
    std::vector<double> oc;
};

// The copies are ordered on the call's stream, so that a new observable does
// not overwrite the one that an earlier asynchronous call on the same stream
// (sd_evolve_observe) has still to read.  Their host sources may be freed on
// return: copies from pageable memory are staged before the call returns.
sd_status stage_obs(sd_ctx *ctx, int64_t mo, const uint64_t *ox, const uint64_t *oz, const double *oc,
                    StagedObs &so, cudaStream_t st) {
    std::vector<uint64_t> dz;
    std::vector<double> dcv;
    so = StagedObs{};
    for (int64_t k = 0; k < mo; k++) {
        if (ox[k] == 0) {
            dz.push_back(oz[k]);
            dcv.push_back(oc[k]);
        } else {
            so.ox.push_back(ox[k]);
            so.oz.push_back(oz[k]);
            so.oc.push_back(oc[k]);
        }
    }
    // full arrays too (for sd_grad's lambda = O phi): layout [dz | dc | ax | az | ac]
    size_t need = dz.size() * 2 + (size_t)mo * 3 + 2;
    if (need > ctx->obs_cap) {
        cudaFree(ctx->d_obs);
        ctx->d_obs = nullptr;
        ctx->obs_cap = 0;
        CK(cudaMalloc((void **)&ctx->d_obs, sizeof(uint64_t) * need));
        ctx->obs_cap = need;
    }
    uint64_t *p = ctx->d_obs;
    so.nd = (int)dz.size();
    so.dz = p;
    so.dc = reinterpret_cast<const double *>(p + dz.size());
    if (!dz.empty()) {
        CK(cudaMemcpyAsync(p, dz.data(), sizeof(uint64_t) * dz.size(), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(p + dz.size(), dcv.data(), sizeof(double) * dcv.size(), cudaMemcpyHostToDevice,
                           st));
    }
    uint64_t *q = p + 2 * dz.size();
    if (mo > 0) {
        CK(cudaMemcpyAsync(q, ox, sizeof(uint64_t) * mo, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(q + mo, oz, sizeof(uint64_t) * mo, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(q + 2 * mo, oc, sizeof(double) * mo, cudaMemcpyHostToDevice, st));
    }
    return SD_OK;
}

const uint64_t *staged_all_x(sd_ctx *ctx, const StagedObs &so) { return ctx->d_obs + 2 * so.nd; }

// <psi|O|psi> into d_out (device), asynchronously.
sd_status expect_async(sd_ctx *ctx, const void *psi, bool dbl, const StagedObs &so, double *d_out,
                       cudaStream_t st) {
    const int blocks = expect_blocks(ctx);
    size_t slots = (size_t)blocks * ((so.nd ? 1 : 0) + so.ox.size());
    sd_status s = ensure_partial(ctx, std::max<size_t>(slots, 1));
    if (s != SD_OK) return s;
    int64_t off = 0;
    if (so.nd) {
        CK(launch_expect_diag(dbl, psi, ctx->n, so.dz, so.dc, so.nd, ctx->d_partial, blocks, st));
        off += blocks;
    }
    for (size_t k = 0; k < so.ox.size(); k++) {
        CK(launch_expect_pauli(dbl, psi, ctx->n, so.ox[k], so.oz[k], so.oc[k], ctx->d_partial + off,
                               blocks, st));
        off += blocks;
    }
    if (off == 0) {
        CK(cudaMemsetAsync(d_out, 0, sizeof(double), st));
        return SD_OK;
    }
    CK(launch_reduce(ctx->d_partial, off, d_out, 0, st));
    return SD_OK;
}

sd_status check_obs(sd_ctx *ctx, int64_t mo, const uint64_t *ox, const uint64_t *oz, const double *oc) {
    if (mo < 0 || (mo > 0 && (!ox || !oz || !oc))) return fail(ctx, SD_EINVAL, "invalid observable arrays");
    const uint64_t lim = (uint64_t(1) << ctx->n) - 1;
    for (int64_t k = 0; k < mo; k++)
        if ((ox[k] & ~lim) || (oz[k] & ~lim) || !std::isfinite(oc[k]))
            return fail(ctx, SD_EINVAL, "observable term " + std::to_string(k) + " is invalid");
    return SD_OK;
}

sd_status get_cliff(sd_ctx *ctx, bool dbl, int g, bool fwd, Program *&out) {
    auto key = std::make_tuple((int)dbl, g, (int)fwd);
    auto it = ctx->cliff_programs.find(key);
    if (it != ctx->cliff_programs.end()) {
        out = it->second.get();
        return SD_OK;
    }
    Circuit c;
    append_clifford(ctx->plan, g, fwd, c);
    auto P = std::make_unique<Program>();
    if (c.ops.empty()) {
        P->onchip = false;   // empty: nothing to run
    } else {
        sd_status s = build_program(ctx, c, dbl, *P);
        if (s != SD_OK) {
            free_program(*P);
            return s;
        }
    }
    out = P.get();
    ctx->cliff_programs[key] = std::move(P);
    return SD_OK;
}

bool program_empty(const Program &P) {
    return P.onchip ? P.circ.n_ops == 0 : P.sched.n_passes == 0;
}

// Program of the change of frame between two group exponentials of the
// adjoint sweep: C_b C_a^dag (leave group a's diagonal frame, enter group
// b's), one circuit so that the one-qubit gates of both merge.
sd_status get_transition(sd_ctx *ctx, bool dbl, int a, int b, Program *&out) {
    auto key = std::make_tuple((int)dbl, a, b);
    auto it = ctx->transition_programs.find(key);
    if (it != ctx->transition_programs.end()) {
        out = it->second.get();
        return SD_OK;
    }
    Circuit c;
    if (a != b) {
        append_clifford(ctx->plan, a, false, c);
        append_clifford(ctx->plan, b, true, c);
    }
    auto P = std::make_unique<Program>();
    if (c.ops.empty()) {
        P->onchip = false;   // empty: nothing to run
    } else {
        sd_status s = build_program(ctx, c, dbl, *P);
        if (s != SD_OK) {
            free_program(*P);
            return s;
        }
    }
    out = P.get();
    ctx->transition_programs[key] = std::move(P);
    return SD_OK;
}

sd_status get_grad_group(sd_ctx *ctx, int g, double f, double dt, GradGroup *&out) {
    auto key = std::make_pair(g, f);
    auto it = ctx->grad_groups.find(key);
    if (it != ctx->grad_groups.end()) {
        out = &it->second;
        return SD_OK;
    }
    const GroupPlan &gp = ctx->plan.groups[g];
    std::vector<std::vector<size_t>> cls(16);
    for (size_t k = 0; k < gp.terms.size(); k++) cls[gp.masks[k] & 15u].push_back(k);
    std::vector<uint64_t> mf;
    std::vector<int64_t> qi;
    std::vector<int32_t> tid;
    std::vector<double> fac;
    GradGroup gg;
    int off = 0;
    const double inv2pi = 1.0 / (2.0 * M_PI);
    for (int s = 0; s < 16; s++) {
        gg.g.off[s] = off;
        for (size_t k : cls[s]) {
            double a = f * dt * ctx->c[gp.terms[k]];
            double sg = gp.signs[k] ? -1.0 : 1.0;
            mf.push_back(gp.masks[k] & ~uint64_t(15));
            qi.push_back((int64_t)(0 - (uint64_t)turns_q64(sg * a * inv2pi)));
            tid.push_back((int32_t)gp.terms[k]);
            fac.push_back(2.0 * f * dt * sg);
            off++;
        }
    }
    gg.g.off[16] = off;
    gg.g.m = off;
    gg.g.base = 0;
    CK(upload(ctx->grad_allocs, gg.masks_f, mf));
    CK(upload(ctx->grad_allocs, gg.qinv, qi));
    CK(upload(ctx->grad_allocs, gg.term_id, tid));
    CK(upload(ctx->grad_allocs, gg.factor, fac));
    ctx->grad_groups[key] = gg;
    out = &ctx->grad_groups[key];
    return SD_OK;
}

}  // namespace

void sd::set_last_error(const std::string &msg) { g_last_error = msg; }

// =================================================================== C ABI

extern "C" {

sd_status sd_create(int n, int64_t m, const uint64_t *xmask, const uint64_t *zmask,
                    const double *coeffs, sd_ctx **out) {
    if (!out) return fail(nullptr, SD_EINVAL, "null output pointer");
    *out = nullptr;
    if (n < 1 || n > 40) return fail(nullptr, SD_EINVAL, "n must be in [1, 40]");
    if (m < 1) return fail(nullptr, SD_EINVAL, "m must be >= 1");
    if (!xmask || !zmask || !coeffs) return fail(nullptr, SD_EINVAL, "null term array");
    const uint64_t lim = (n >= 64) ? ~uint64_t(0) : ((uint64_t(1) << n) - 1);
    for (int64_t j = 0; j < m; j++) {
        if ((xmask[j] & ~lim) || (zmask[j] & ~lim))
            return fail(nullptr, SD_EINVAL, "term " + std::to_string(j) + " has a mask bit >= n");
        if (!std::isfinite(coeffs[j]))
            return fail(nullptr, SD_EINVAL, "term " + std::to_string(j) + " has a non-finite coefficient");
    }
    sd_ctx *ctx = new (std::nothrow) sd_ctx;
    if (!ctx) return fail(nullptr, SD_ENOMEM, "out of host memory");
    ctx->n = n;
    ctx->m = m;
    ctx->x.assign(xmask, xmask + m);
    ctx->z.assign(zmask, zmask + m);
    ctx->c.assign(coeffs, coeffs + m);
    *out = ctx;
    return SD_OK;
}

sd_status sd_create_str(int n, int64_t m, const char *const *paulis, const double *coeffs,
                        sd_ctx **out) {
    if (!out) return fail(nullptr, SD_EINVAL, "null output pointer");
    *out = nullptr;
    if (!paulis || m < 1 || n < 1 || n > 40) return fail(nullptr, SD_EINVAL, "invalid arguments");
    std::vector<uint64_t> x(m, 0), z(m, 0);
    for (int64_t j = 0; j < m; j++) {
        const char *s = paulis[j];
        if (!s || (int)strlen(s) != n)
            return fail(nullptr, SD_EINVAL, "string " + std::to_string(j) + " does not have length n");
        for (int q = 0; q < n; q++) {
            char ch = s[q];
            if (ch >= 'a' && ch <= 'z') ch = char(ch - 'a' + 'A');
            uint64_t b = uint64_t(1) << q;
            if (ch == 'X') x[j] |= b;
            else if (ch == 'Z') z[j] |= b;
            else if (ch == 'Y') { x[j] |= b; z[j] |= b; }
            else if (ch != 'I')
                return fail(nullptr, SD_EINVAL, "string " + std::to_string(j) + " has a character outside IXYZ");
        }
    }
    return sd_create(n, m, x.data(), z.data(), coeffs, out);
}

sd_status sd_set_coeffs(sd_ctx *ctx, const double *coeffs) {
    if (!ctx || !coeffs) return fail(ctx, SD_EINVAL, "null argument");
    for (int64_t j = 0; j < ctx->m; j++)
        if (!std::isfinite(coeffs[j]))
            return fail(ctx, SD_EINVAL, "term " + std::to_string(j) + " has a non-finite coefficient");
    ctx->c.assign(coeffs, coeffs + ctx->m);
    batch_purge(ctx);
    for (auto &kv : ctx->programs) free_program(*kv.second);
    ctx->programs.clear();
    for (void *p : ctx->grad_allocs) cudaFree(p);
    ctx->grad_allocs.clear();
    ctx->grad_groups.clear();
    return SD_OK;
}

sd_status sd_plan(sd_ctx *ctx, const sd_plan_opts *opts) {
    if (!ctx) return fail(nullptr, SD_EINVAL, "null context");
    int rule = 2, tb = 0, jit = 0, grouping = 0, layout = 0, prefetch = 0;
    if (opts) {
        rule = opts->skip_rule < 0 ? 2 : opts->skip_rule;
        tb = opts->tile_bits;
        jit = opts->jit;
        grouping = opts->grouping;
        layout = opts->layout;
        prefetch = opts->prefetch;
        if (layout < -1 || layout > 1) return fail(ctx, SD_EINVAL, "layout must be -1, 0 or 1");
        if (prefetch < 0 || prefetch > 3) return fail(ctx, SD_EINVAL, "prefetch must be 0, 1, 2 or 3");
        if (rule > 2) return fail(ctx, SD_EINVAL, "skip_rule must be -1, 0, 1 or 2");
        if (tb != 0 && (tb < 9 || tb > 13)) return fail(ctx, SD_EINVAL, "tile_bits must be 0 or 9..13");
        if (grouping < 0 || grouping > 3) return fail(ctx, SD_EINVAL, "grouping must be 0, 1, 2 or 3");
    }
    Plan p;
    std::string e = make_plan(ctx->n, ctx->m, ctx->x.data(), ctx->z.data(), rule, p, grouping, ctx->c.data());
    if (!e.empty()) return fail(ctx, SD_EINTERNAL, "planner: " + e);
    batch_purge(ctx);
    for (auto &kv : ctx->programs) free_program(*kv.second);
    ctx->programs.clear();
    for (auto &kv : ctx->cliff_programs) free_program(*kv.second);
    ctx->cliff_programs.clear();
    for (auto &kv : ctx->transition_programs) free_program(*kv.second);
    ctx->transition_programs.clear();
    for (void *a : ctx->grad_allocs) cudaFree(a);
    ctx->grad_allocs.clear();
    ctx->grad_groups.clear();
    ctx->plan = std::move(p);
    ctx->tile_bits_opt = tb;
    ctx->tuned_k[0] = ctx->tuned_k[1] = 0;
    ctx->jit_opt = jit;
    ctx->layout_opt = layout;
    ctx->tuned_layout = 0;
    ctx->prefetch_opt = prefetch;
    ctx->tuned_prefetch[0] = ctx->tuned_prefetch[1] = 0;
    ctx->planned = true;
    // plan view
    ctx->v_goff.assign(1, 0);
    ctx->v_gterms.clear();
    ctx->v_masks.clear();
    ctx->v_signs.clear();
    ctx->v_gateoff.assign(1, 0);
    ctx->v_gates.clear();
    ctx->v_cols.clear();
    ctx->v_icols.clear();
    for (auto &g : ctx->plan.groups) {
        for (size_t k = 0; k < g.terms.size(); k++) {
            ctx->v_gterms.push_back(g.terms[k]);
            ctx->v_masks.push_back(g.masks[k]);
            ctx->v_signs.push_back(g.signs[k]);
        }
        ctx->v_goff.push_back((int64_t)ctx->v_gterms.size());
        for (auto &gt : g.gates) {
            ctx->v_gates.push_back(gt.kind);
            ctx->v_gates.push_back(gt.a);
            ctx->v_gates.push_back(gt.b);
        }
        ctx->v_gateoff.push_back((int64_t)ctx->v_gates.size() / 3);
        ctx->v_cols.insert(ctx->v_cols.end(), g.cnot_cols.begin(), g.cnot_cols.end());
        ctx->v_icols.insert(ctx->v_icols.end(), g.cnot_inv_cols.begin(), g.cnot_inv_cols.end());
    }
    return SD_OK;
}

sd_status sd_get_plan(const sd_ctx *ctx, sd_plan_view *out) {
    if (!ctx || !out) return fail(nullptr, SD_EINVAL, "null argument");
    if (!ctx->planned) return fail(const_cast<sd_ctx *>(ctx), SD_ENOPLAN, "sd_plan has not been called");
    out->n = ctx->n;
    out->m = ctx->m;
    out->n_groups = (int64_t)ctx->plan.groups.size();
    out->group_offsets = ctx->v_goff.data();
    out->group_terms = ctx->v_gterms.data();
    out->masks = ctx->v_masks.data();
    out->signs = ctx->v_signs.data();
    out->gate_offsets = ctx->v_gateoff.data();
    out->gates = ctx->v_gates.data();
    out->cnot_cols = ctx->v_cols.data();
    out->cnot_inv_cols = ctx->v_icols.data();
    return SD_OK;
}

sd_status sd_get_schedule(sd_ctx *ctx, sd_dtype dtype, int order, sd_schedule_stats *out) {
    if (!ctx || !out) return fail(nullptr, SD_EINVAL, "null argument");
    if (!ctx->planned) return fail(ctx, SD_ENOPLAN, "sd_plan has not been called");
    if (order != 1 && order != 2) return fail(ctx, SD_EINVAL, "order must be 1 or 2");
    const bool dbl = dtype == SD_C128;
    memset(out, 0, sizeof(*out));
    out->onchip = use_onchip(ctx, dbl) ? 1 : 0;
    if (out->onchip) return SD_OK;
    const int G = (int)ctx->plan.groups.size();
    Circuit c = segment_circuit(ctx, order, (order == 2 && G > 1) ? 2 : 0, 0.01);
    canonicalize_1q(c, ctx->n);
    Schedule S;   // as sd_evolve schedules it (smaller tiles if a pass's terms need the room)
    sd_status s = schedule_for(ctx, c, dbl, S, pin0_wanted(ctx, dbl, true));
    if (s != SD_OK) return s;
    out->tile_bits = S.K;
    out->passes_per_step = (int64_t)S.passes.size();
    out->rounds_per_step = (int64_t)S.rounds.size();
    out->diag_passes = S.diag_passes;
    return SD_OK;
}

sd_status sd_prepare(sd_ctx *ctx, sd_dtype dtype, double dt, int64_t steps, int order) {
    if (!ctx) return fail(nullptr, SD_EINVAL, "null context");
    if (!ctx->planned) return fail(ctx, SD_ENOPLAN, "sd_plan has not been called");
    if (dtype != SD_C64 && dtype != SD_C128) return fail(ctx, SD_EINVAL, "dtype must be SD_C64 or SD_C128");
    if (order != 1 && order != 2) return fail(ctx, SD_EINVAL, "order must be 1 or 2");
    if (steps < 0) return fail(ctx, SD_EINVAL, "steps must be >= 0");
    if (!std::isfinite(dt)) return fail(ctx, SD_EINVAL, "dt must be finite");
    sd_status s = ensure_device(ctx);
    if (s != SD_OK || steps == 0) return s;
    return evolve_impl(ctx, nullptr, dtype == SD_C128, dt, steps, order, nullptr, false);
}

namespace {

// Times sd_evolve(., dt, steps, order) on a scratch state for every tile size
// K = kmin..kmax and every layout of `layouts` (complex64 only: -1 plain,
// 1 paired), after one untimed call that builds and compiles the programs;
// keeps the fastest pair for the dtype.  ms[l][K - 9] receives ms per step.
sd_status autotune_impl(sd_ctx *ctx, sd_dtype dtype, double dt, int64_t steps, int order, int kmin, int kmax,
                        const std::vector<std::pair<int, int>> &shapes, int *best_k, int *best_layout,
                        int *best_prefetch, double ms[4][5]) {
    if (!ctx) return fail(nullptr, SD_EINVAL, "null context");
    if (!ctx->planned) return fail(ctx, SD_ENOPLAN, "sd_plan has not been called");
    if (dtype != SD_C64 && dtype != SD_C128) return fail(ctx, SD_EINVAL, "dtype must be SD_C64 or SD_C128");
    if (order != 1 && order != 2) return fail(ctx, SD_EINVAL, "order must be 1 or 2");
    if (steps < 1 || !std::isfinite(dt)) return fail(ctx, SD_EINVAL, "steps must be >= 1 and dt finite");
    if (kmin < kRegBits + kLaneBits || kmax > 13 || kmin > kmax)
        return fail(ctx, SD_EINVAL, "tile sizes must satisfy 9 <= kmin <= kmax <= 13");
    const bool dbl = dtype == SD_C128;
    const int d = dbl ? 1 : 0;
    for (int l = 0; l < 4; l++)
        for (int k = 0; k < 5; k++) ms[l][k] = 0.0;
    *best_k = 0;
    *best_layout = 0;
    *best_prefetch = 0;
    sd_status s = ensure_device(ctx);
    if (s != SD_OK) return s;
    if (use_onchip(ctx, dbl)) return SD_OK;   // nothing to tune: one launch runs every step
    auto drop_programs = [&]() {
        batch_purge(ctx);
        for (auto &kv : ctx->programs) free_program(*kv.second);
        ctx->programs.clear();
    };
    const size_t bytes = ((size_t)1 << ctx->n) * (dbl ? 16 : 8);
    void *scratch = nullptr;
    if (cudaMalloc(&scratch, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, SD_ENOMEM, "no device memory for the autotuner's scratch state");
    }
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const int saved = ctx->tuned_k[d], saved_layout = ctx->tuned_layout, saved_pf = ctx->tuned_prefetch[d];
    int best = 0, best_l = 0, best_pf = 0;
    double best_ms = 0.0;
    s = SD_OK;
    cudaError_t ce = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(scratch, 0, bytes, st);
    if (ce != cudaSuccess) s = fail(ctx, SD_ECUDA, std::string("autotune: ") + cudaGetErrorString(ce));
    for (const auto &shape : shapes) {
        const int L = shape.first, PF = shape.second;
        if (!dbl) ctx->tuned_layout = L;
        ctx->tuned_prefetch[d] = PF;
        for (int K = kmin; K <= kmax && s == SD_OK; K++) {
            if (K > ctx->n) break;
            ctx->tuned_k[d] = K;
            drop_programs();
            // warm-up call of the timed shape (builds and compiles its programs)
            sd_status r = evolve_impl(ctx, scratch, dbl, dt, steps, order, st);
            if (r == SD_OK && cudaStreamSynchronize(st) != cudaSuccess) r = SD_ECUDA;
            if (r != SD_OK) {
                // a tile size the scheduler or the device cannot run is skipped
                cudaGetLastError();
                continue;
            }
            cudaEventRecord(e0, st);
            r = evolve_impl(ctx, scratch, dbl, dt, steps, order, st);
            cudaEventRecord(e1, st);
            if (r != SD_OK || cudaEventSynchronize(e1) != cudaSuccess) {
                s = fail(ctx, SD_ECUDA, "autotune: timed run failed");
                break;
            }
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            const double per = (double)t / (double)steps;
            ms[(L > 0 ? 2 : 0) + (PF > 1 ? 1 : 0)][K - 9] = per;
            if (best == 0 || per < best_ms) {
                best = K;
                best_l = L;
                best_pf = PF;
                best_ms = per;
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    cudaFree(scratch);
    const bool ok = s == SD_OK && best > 0;
    ctx->tuned_k[d] = ok ? best : saved;
    if (!dbl) ctx->tuned_layout = ok ? best_l : saved_layout;
    ctx->tuned_prefetch[d] = ok ? best_pf : saved_pf;
    drop_programs();
    if (s != SD_OK) return s;
    if (best == 0) return fail(ctx, SD_EINVAL, "no tile size in the range could be scheduled");
    *best_k = best;
    *best_layout = best_l;
    *best_prefetch = best_pf;
    return SD_OK;
}

}  // namespace

sd_status sd_autotune(sd_ctx *ctx, sd_dtype dtype, double dt, int64_t steps, int order, int kmin, int kmax,
                      int *best_k, double *times_ms) {
    int bk = 0, bl = 0, bp = 0;
    double ms[4][5];
    // the layout and prefetch depth in force (sd_plan's, else the tuned ones,
    // else plain and one buffer) are kept
    int L = -1, PF = 1;
    if (ctx) {
        L = ctx->layout_opt != 0 ? ctx->layout_opt : (ctx->tuned_layout != 0 ? ctx->tuned_layout : -1);
        PF = prefetch_buffers(ctx, dtype == SD_C128);
    }
    if (times_ms && kmin <= kmax)
        for (int k = kmin; k <= kmax; k++) times_ms[k - kmin] = 0.0;
    if (best_k) *best_k = 0;
    sd_status s = autotune_impl(ctx, dtype, dt, steps, order, kmin, kmax, {{L, PF}}, &bk, &bl, &bp, ms);
    if (s != SD_OK) return s;
    if (times_ms)
        for (int k = kmin; k <= kmax; k++) times_ms[k - kmin] = ms[(L > 0 ? 2 : 0) + (PF > 1 ? 1 : 0)][k - 9];
    if (best_k) *best_k = bk;
    return SD_OK;
}

sd_status sd_autotune_shape(sd_ctx *ctx, sd_dtype dtype, double dt, int64_t steps, int order, int kmin,
                            int kmax, sd_tune_result *out) {
    if (!out) return fail(ctx, SD_EINVAL, "null result pointer");
    memset(out, 0, sizeof(*out));
    // the paired layout exists for complex64 passes compiled at run time, the
    // second prefetch buffer for passes compiled at run time; options given
    // to sd_plan are kept
    std::vector<int> layouts{-1}, depths{1};
    const bool jit = ctx && jit_wanted(ctx, true, 1);
    if (ctx && dtype == SD_C64 && ctx->layout_opt != 0) layouts.assign(1, ctx->layout_opt);
    else if (dtype == SD_C64 && jit) layouts.push_back(1);
    if (ctx && ctx->prefetch_opt != 0) depths.assign(1, ctx->prefetch_opt);
    else if (jit) depths.push_back(two_buffer_form(dtype == SD_C128));
    std::vector<std::pair<int, int>> shapes;
    for (int L : layouts)
        for (int PF : depths) shapes.push_back({L, PF});
    return autotune_impl(ctx, dtype, dt, steps, order, kmin, kmax, shapes, &out->best_k, &out->best_layout,
                         &out->best_prefetch, out->ms);
}

sd_status sd_evolve_host(sd_ctx *ctx, void *host_state, void *d_work, sd_dtype dtype, double dt,
                         int64_t steps, int order, void *cuda_stream) {
    sd_status s = check_state_args(ctx, d_work, dtype, order);
    if (s != SD_OK) return s;
    if (!host_state) return fail(ctx, SD_EINVAL, "null host state");
    if (steps < 0 || !std::isfinite(dt)) return fail(ctx, SD_EINVAL, "invalid steps or dt");
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, host_state) != cudaSuccess || at.type != cudaMemoryTypeHost) {
        cudaGetLastError();
        return fail(ctx, SD_EINVAL, "host state must be page-locked host memory (cudaHostAlloc, cudaHostRegister)");
    }
    const bool dbl = dtype == SD_C128;
    const size_t bytes = ((size_t)1 << ctx->n) * (dbl ? 16 : 8);
    void *hp = at.devicePointer ? at.devicePointer : host_state;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    CK(launch_copy16(hp, d_work, bytes, ctx->num_sms, st));
    if (steps > 0 && (s = evolve_impl(ctx, d_work, dbl, dt, steps, order, st)) != SD_OK) return s;
    CK(launch_copy16(d_work, hp, bytes, ctx->num_sms, st));
    return SD_OK;
}

sd_status sd_precompile(sd_ctx *ctx, sd_dtype dtype, int64_t steps, int order, int64_t *compiled) {
    if (!ctx) return fail(nullptr, SD_EINVAL, "null context");
    if (!ctx->planned) return fail(ctx, SD_ENOPLAN, "sd_plan has not been called");
    if (dtype != SD_C64 && dtype != SD_C128) return fail(ctx, SD_EINVAL, "dtype must be SD_C64 or SD_C128");
    if (order != 1 && order != 2) return fail(ctx, SD_EINVAL, "order must be 1 or 2");
    if (steps < 0) return fail(ctx, SD_EINVAL, "steps must be >= 0");
    if (compiled) *compiled = 0;
    const bool dbl = dtype == SD_C128;
    if (steps == 0 || use_onchip(ctx, dbl)) return SD_OK;
    const int G = (int)ctx->plan.groups.size();
    // the segments sd_evolve would run: (kind, repetitions in one program)
    std::vector<std::pair<int, int>> segs;
    int64_t one = 0;
    sd_status s;
    const int base = (order == 1 || G == 1 || steps == 1) ? 0 : 2;
    const int64_t count = base == 0 ? steps : steps - 1;
    if (base == 2) {
        segs.push_back({1, 1});
        segs.push_back({3, 1});
    }
    if ((s = segment_passes(ctx, dbl, order, base, 1, one)) != SD_OK) return s;
    const int M = block_steps(one);
    if (count > 0 && (count % M != 0 || M == 1)) segs.push_back({base, 1});
    if (M > 1 && count >= M) segs.push_back({4, M});
    int64_t total = 0;
    for (auto &sg : segs) {
        Circuit c = segment_circuit(ctx, order, sg.first, 0.01, sg.second);
        canonicalize_1q(c, ctx->n);
        Schedule S;
        const bool allow = sg.first != 1;
        if ((s = schedule_for(ctx, c, dbl, S, pin0_wanted(ctx, dbl, allow))) != SD_OK) return s;
        S.prefetch = prefetch_buffers(ctx, dbl);
        if (!jit_wanted(ctx, allow, (int64_t)S.passes.size())) continue;
        int done = 0;
        const std::string e = jit_precompile(S, ctx->n, dbl, &done);
        if (!e.empty()) return fail(ctx, SD_EINVAL, "run-time compilation: " + e);
        total += done;
    }
    if (compiled) *compiled = total;
    return SD_OK;
}

sd_status sd_count_passes(sd_ctx *ctx, sd_dtype dtype, int order, int64_t steps, int64_t *out) {
    if (!ctx || !out) return fail(nullptr, SD_EINVAL, "null argument");
    if (!ctx->planned) return fail(ctx, SD_ENOPLAN, "sd_plan has not been called");
    if (order != 1 && order != 2) return fail(ctx, SD_EINVAL, "order must be 1 or 2");
    if (dtype != SD_C64 && dtype != SD_C128) return fail(ctx, SD_EINVAL, "dtype must be SD_C64 or SD_C128");
    if (steps < 0) return fail(ctx, SD_EINVAL, "steps must be >= 0");
    *out = 0;
    const bool dbl = dtype == SD_C128;
    if (steps == 0 || use_onchip(ctx, dbl)) return SD_OK;
    const int G = (int)ctx->plan.groups.size();
    sd_status s;
    auto repeated = [&](int kind, int64_t count, int64_t &total) -> sd_status {
        int64_t one = 0, blk = 0;
        sd_status r = segment_passes(ctx, dbl, order, kind, 1, one);
        if (r != SD_OK) return r;
        const int M = block_steps(one);
        if (M > 1 && count >= M) {
            if ((r = segment_passes(ctx, dbl, order, 4, M, blk)) != SD_OK) return r;
            total += (count / M) * blk;
            count %= M;
        }
        total += count * one;
        return SD_OK;
    };
    int64_t total = 0;
    if (order == 1 || G == 1 || steps == 1) {
        if ((s = repeated(0, steps, total)) != SD_OK) return s;
    } else {
        int64_t h = 0, t = 0;
        if ((s = segment_passes(ctx, dbl, order, 1, 1, h)) != SD_OK) return s;
        if ((s = segment_passes(ctx, dbl, order, 3, 1, t)) != SD_OK) return s;
        if ((s = repeated(2, steps - 1, total)) != SD_OK) return s;
        total += h + t;
    }
    *out = total;
    return SD_OK;
}

sd_status sd_evolve(sd_ctx *ctx, void *d_state, sd_dtype dtype, double dt, int64_t steps, int order,
                    void *cuda_stream) {
    sd_status s = check_state_args(ctx, d_state, dtype, order);
    if (s != SD_OK) return s;
    if (steps < 0) return fail(ctx, SD_EINVAL, "steps must be >= 0");
    if (!std::isfinite(dt)) return fail(ctx, SD_EINVAL, "dt must be finite");
    if (steps == 0) return SD_OK;
    return evolve_impl(ctx, d_state, dtype == SD_C128, dt, steps, order, (cudaStream_t)cuda_stream);
}


sd_status sd_evolve_observe(sd_ctx *ctx, void *d_state, sd_dtype dtype, double dt, int64_t steps,
                            int order, int64_t mo, const uint64_t *ox, const uint64_t *oz,
                            const double *oc, double *d_trace, void *cuda_stream) {
    sd_status s = check_state_args(ctx, d_state, dtype, order);
    if (s != SD_OK) return s;
    if (steps < 0 || !std::isfinite(dt)) return fail(ctx, SD_EINVAL, "invalid steps or dt");
    if ((s = check_obs(ctx, mo, ox, oz, oc)) != SD_OK) return s;
    if (steps > 0 && !d_trace) return fail(ctx, SD_EINVAL, "null trace pointer");
    if (steps == 0) return SD_OK;
    const bool dbl = dtype == SD_C128;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    StagedObs so;
    if ((s = stage_obs(ctx, mo, ox, oz, oc, so, st)) != SD_OK) return s;
    Program *P = nullptr;
    if ((s = get_program(ctx, dbl, order, 0, dt, P)) != SD_OK) return s;
    if (P->onchip && so.ox.empty())
        return run_program(ctx, dbl, *P, d_state, steps, st, so.dz, so.dc, so.nd, d_trace);
    for (int64_t k = 0; k < steps; k++) {
        if ((s = run_program(ctx, dbl, *P, d_state, 1, st)) != SD_OK) return s;
        if ((s = expect_async(ctx, d_state, dbl, so, d_trace + k, st)) != SD_OK) return s;
    }
    return SD_OK;
}

sd_status sd_evolve_pauli(sd_ctx *ctx, void *d_state, sd_dtype dtype, double dt, int64_t steps,
                          int order, void *cuda_stream) {
    sd_status s = check_state_args(ctx, d_state, dtype, order);
    if (s != SD_OK) return s;
    if (steps < 0 || !std::isfinite(dt)) return fail(ctx, SD_EINVAL, "invalid steps or dt");
    const bool dbl = dtype == SD_C128;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int G = (int)ctx->plan.groups.size();
    std::vector<std::pair<int64_t, double>> seq;   // (term, angle)
    for (auto &p : step_sequence(G, order))
        for (int64_t j : ctx->plan.groups[p.first].terms) seq.push_back({j, p.second * dt * ctx->c[j]});
    for (int64_t k = 0; k < steps; k++)
        for (auto &t : seq)
            CK(launch_pauli_rotation(dbl, d_state, ctx->n, ctx->x[t.first], ctx->z[t.first],
                                     std::cos(t.second), std::sin(t.second), ctx->num_sms, st));
    return SD_OK;
}

sd_status sd_expect(sd_ctx *ctx, const void *d_state, sd_dtype dtype, int64_t mo, const uint64_t *ox,
                    const uint64_t *oz, const double *oc, double *out_host, void *cuda_stream) {
    if (!out_host) return fail(ctx, SD_EINVAL, "null output pointer");
    sd_status s = check_state_args(ctx, d_state, dtype, 1);
    if (s != SD_OK) return s;
    if ((s = check_obs(ctx, mo, ox, oz, oc)) != SD_OK) return s;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    StagedObs so;
    if ((s = stage_obs(ctx, mo, ox, oz, oc, so, st)) != SD_OK) return s;
    if ((s = ensure_partial(ctx, 1)) != SD_OK) return s;
    if ((s = expect_async(ctx, d_state, dtype == SD_C128, so, ctx->d_scalar, st)) != SD_OK) return s;
    double v = 0.0;
    CK(cudaMemcpyAsync(&v, ctx->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *out_host = v;
    return SD_OK;
}

sd_status sd_grad(sd_ctx *ctx, const void *d_state0, sd_dtype dtype, double dt, int64_t steps,
                  int order, int64_t mo, const uint64_t *ox, const uint64_t *oz, const double *oc,
                  double *value_out, double *grad_out, void *cuda_stream) {
    sd_status s = check_state_args(ctx, d_state0, dtype, order);
    if (s != SD_OK) return s;
    if (!value_out || !grad_out) return fail(ctx, SD_EINVAL, "null output pointer");
    if (steps < 0 || !std::isfinite(dt)) return fail(ctx, SD_EINVAL, "invalid steps or dt");
    if (ctx->n < 4) return fail(ctx, SD_EINVAL, "sd_grad needs n >= 4");
    if ((s = check_obs(ctx, mo, ox, oz, oc)) != SD_OK) return s;
    const bool dbl = dtype == SD_C128;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const size_t bytes = (size_t)(dbl ? 16 : 8) << ctx->n;
    if (ctx->work_bytes < bytes) {
        cudaFree(ctx->d_work[0]);
        cudaFree(ctx->d_work[1]);
        ctx->d_work[0] = ctx->d_work[1] = nullptr;
        ctx->work_bytes = 0;
        CK(cudaMalloc(&ctx->d_work[0], bytes));
        CK(cudaMalloc(&ctx->d_work[1], bytes));
        ctx->work_bytes = bytes;
    }
    if (!ctx->d_gacc) CK(cudaMalloc((void **)&ctx->d_gacc, sizeof(double) * std::max<int64_t>(ctx->m, 1)));
    // gradient programs depend on dt: drop those made for another step size
    if (!ctx->grad_groups.empty() && ctx->grad_dt != dt) {
        for (void *a : ctx->grad_allocs) cudaFree(a);
        ctx->grad_allocs.clear();
        ctx->grad_groups.clear();
    }
    ctx->grad_dt = dt;
    void *phi = ctx->d_work[0], *lam = ctx->d_work[1];
    CK(cudaMemcpyAsync(phi, d_state0, bytes, cudaMemcpyDeviceToDevice, st));
    if ((s = evolve_impl(ctx, phi, dbl, dt, steps, order, st)) != SD_OK) return s;
    StagedObs so;
    if ((s = stage_obs(ctx, mo, ox, oz, oc, so, st)) != SD_OK) return s;
    if ((s = ensure_partial(ctx, 1)) != SD_OK) return s;
    if ((s = expect_async(ctx, phi, dbl, so, ctx->d_scalar, st)) != SD_OK) return s;
    const uint64_t *ax = staged_all_x(ctx, so);
    CK(launch_apply_observable(dbl, phi, lam, ctx->n, ax, ax + mo,
                               reinterpret_cast<const double *>(ax + 2 * mo), (int)mo, st));
    CK(cudaMemsetAsync(ctx->d_gacc, 0, sizeof(double) * ctx->m, st));
    const int G = (int)ctx->plan.groups.size();
    const int blocks = grad_blocks(ctx->n, ctx->num_sms);
    auto seq = step_sequence(G, order);
    DevTables tabs;   // e^{2 pi i k/256} for the adjoint kernel's rotations
    if ((s = device_tables(ctx, tabs)) != SD_OK) return s;
    // Reverse sweep over the group exponentials.  phi and lam stay in the
    // diagonal frame of the exponential at hand: C_g brings them into the
    // first one's, each change of group runs one merged program C_b C_a^dag,
    // and no frame is left at the end (only the gradient is kept).
    int prev = -1;
    for (int64_t k = 0; k < steps; k++) {
        for (auto it = seq.rbegin(); it != seq.rend(); ++it) {
            const int g = it->first;
            Program *tr = nullptr;
            GradGroup *gg = nullptr;
            if (prev < 0) s = get_cliff(ctx, dbl, g, true, tr);
            else s = get_transition(ctx, dbl, prev, g, tr);
            if (s != SD_OK) return s;
            if ((s = get_grad_group(ctx, g, it->second, dt, gg)) != SD_OK) return s;
            if ((s = ensure_partial(ctx, (size_t)blocks * std::max(gg->g.m, 1))) != SD_OK) return s;
            if (!program_empty(*tr)) {
                if ((s = run_program(ctx, dbl, *tr, phi, 1, st)) != SD_OK) return s;
                if ((s = run_program(ctx, dbl, *tr, lam, 1, st)) != SD_OK) return s;
            }
            CK(launch_grad_diag(dbl, phi, lam, ctx->n, gg->g, gg->masks_f, gg->qinv, tabs.fxt,
                                ctx->d_partial, blocks, st));
            CK(launch_grad_finalize(ctx->d_partial, blocks, gg->g.m, gg->term_id, gg->factor,
                                    ctx->d_gacc, st));
            prev = g;
        }
    }
    double v = 0.0;
    CK(cudaMemcpyAsync(&v, ctx->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(grad_out, ctx->d_gacc, sizeof(double) * ctx->m, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *value_out = v;
    return SD_OK;
}

}  // extern "C"

namespace {

// ------------------------------------------------------------ batch descriptors
// The device descriptors of an sd_evolve_batch call (each instance's
// programs and share of blocks) are kept for reuse, so that a repeated call
// copies nothing from the host and can be captured in a CUDA graph.  An
// entry refers to its instances' programs, so it is dropped whenever one of
// those contexts frees programs (another dt, new coefficients, a new plan,
// sd_destroy).
struct BatchGroup {
    int K;
    size_t smem;
    int ctas;
    int64_t levels;
    BatchInstance *d_inst;
    uint16_t *d_cta;
};
struct BatchEntry {
    std::vector<sd_ctx *> ctxs;
    std::vector<void *> states;
    int dtype;
    double dt;
    int64_t steps;
    int order;
    std::vector<int64_t> alone;   // instances run like sd_evolve (on chip, large, or mixed tile sizes)
    std::vector<BatchGroup> groups;
    // Streams on which the instances that run alone proceed side by side with
    // each other and with the level launches, forked from and joined back to
    // the caller's stream by events (also inside a stream capture).
    std::vector<cudaStream_t> side;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
};
// Side streams of a batch: at most this many.
constexpr size_t kBatchSideStreams = 8;
std::recursive_mutex g_batch_mu;
// An instance with 2^8 or more tiles (a tile per SM at least) runs on its own.
constexpr int kBatchAloneTileBits = 8;
std::list<BatchEntry> g_batches;   // most recent first
constexpr size_t kBatchCache = 8;

void free_batch(BatchEntry &e) {
    for (auto &g : e.groups) {
        cudaFree(g.d_inst);
        cudaFree(g.d_cta);
    }
    for (cudaStream_t x : e.side) cudaStreamDestroy(x);
    for (cudaEvent_t x : e.join) cudaEventDestroy(x);
    if (e.fork) cudaEventDestroy(e.fork);
    e.side.clear();
    e.join.clear();
    e.fork = nullptr;
}

void batch_purge(const sd_ctx *ctx) {
    std::lock_guard<std::recursive_mutex> lk(g_batch_mu);
    for (auto it = g_batches.begin(); it != g_batches.end();) {
        if (std::find(it->ctxs.begin(), it->ctxs.end(), ctx) != it->ctxs.end()) {
            free_batch(*it);
            it = g_batches.erase(it);
        } else {
            ++it;
        }
    }
}

// Finds or builds the descriptors of a batch call (programs included).
// Building allocates and copies synchronously, so it is refused while `st`
// is being captured.  Called with g_batch_mu held.
sd_status batch_entry(sd_ctx *const *ctxs, void *const *d_states, int64_t count, sd_dtype dtype, double dt,
                      int64_t steps, int order, cudaStream_t st, BatchEntry *&out) {
    const bool dbl = dtype == SD_C128;
    struct Item {
        sd_ctx *ctx;
        void *psi;
        Program *prog[3];
        int64_t reps;
        int64_t index;
    };
    std::vector<Item> items;
    for (int64_t i = 0; i < count; i++) {
        sd_ctx *ctx = ctxs[i];
        const int G = (int)ctx->plan.groups.size();
        Item it{ctx, d_states[i], {nullptr, nullptr, nullptr}, steps, i};
        sd_status s;
        if (order == 1 || G == 1 || steps == 1) {
            if ((s = get_program(ctx, dbl, order, 0, dt, it.prog[1])) != SD_OK) return s;
        } else {
            if ((s = get_program(ctx, dbl, order, 1, dt, it.prog[0])) != SD_OK) return s;
            if ((s = get_program(ctx, dbl, order, 2, dt, it.prog[1])) != SD_OK) return s;
            if ((s = get_program(ctx, dbl, order, 3, dt, it.prog[2])) != SD_OK) return s;
            it.reps = steps - 1;
        }
        items.push_back(it);
    }
    for (auto &e : g_batches)
        if (e.dtype == (int)dtype && e.dt == dt && e.steps == steps && e.order == order &&
            e.ctxs.size() == (size_t)count && std::equal(e.ctxs.begin(), e.ctxs.end(), ctxs) &&
            std::equal(e.states.begin(), e.states.end(), d_states)) {
            out = &e;
            return SD_OK;
        }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) == cudaSuccess && cap != cudaStreamCaptureStatusNone)
        return fail(ctxs[0], SD_EINVAL,
                    "sd_evolve_batch under stream capture needs its descriptors built first: call "
                    "sd_prepare_batch (or the same sd_evolve_batch) outside the capture");
    BatchEntry e;
    e.ctxs.assign(ctxs, ctxs + count);
    e.states.assign(d_states, d_states + count);
    e.dtype = (int)dtype;
    e.dt = dt;
    e.steps = steps;
    e.order = order;
    std::map<int, std::vector<Item>> by_k;
    for (auto &it : items) {
        int K = -1;
        bool mixed = false;
        for (Program *p : it.prog) {
            if (!p) continue;
            if (p->onchip) mixed = true;
            else if (K < 0) K = p->sched.K;
            else if (K != p->sched.K) mixed = true;
        }
        // Instances large enough to fill the GPU on their own run like
        // sd_evolve, with their passes compiled at run time; the rest share
        // the level launches of the interpreter kernel.
        if (mixed || K < 0 || (it.ctx->n - K >= kBatchAloneTileBits && jit_wanted(it.ctx, true, it.prog[1]->passes))) {
            // run like sd_evolve; build its block programs now
            sd_status s = evolve_impl(it.ctx, it.psi, dbl, dt, steps, order, st, false);
            if (s != SD_OK) return s;
            e.alone.push_back(it.index);
        } else {
            by_k[K].push_back(it);
        }
    }
    for (auto &kv : by_k) {
        const int K = kv.first;
        std::vector<Item> &grp = kv.second;
        sd_ctx *ctx = grp[0].ctx;
        int64_t total_tiles = 0;
        size_t smem = 0;
        for (auto &it : grp) {
            total_tiles += (int64_t)1 << (it.ctx->n - K);
            for (Program *p : it.prog)
                if (p)
                    for (auto &ps : p->sched.host_passes) smem = std::max(smem, pass_smem_bytes(ps, dbl ? 16 : 8, K));
        }
        if (smem > kTileSmemLimit) return fail(ctx, SD_EINTERNAL, "batch pass needs too much shared memory");
        const int occ = tile_pass_batch_occupancy(dbl, K, smem);
        const int64_t target = (int64_t)ctx->num_sms * occ * 2;
        std::vector<BatchInstance> inst(grp.size());
        std::vector<uint16_t> cta;
        int64_t max_levels = 0;
        for (size_t i = 0; i < grp.size(); i++) {
            const Item &it = grp[i];
            const int64_t tiles = (int64_t)1 << (it.ctx->n - K);
            int64_t c = (target * tiles + total_tiles - 1) / total_tiles;
            c = std::max<int64_t>(1, std::min(c, tiles));
            BatchInstance &B = inst[i];
            B.psi = it.psi;
            B.n = it.ctx->n;
            B.cta_begin = (int)cta.size();
            B.cta_count = (int)c;
            B.reps_core = it.reps;
            for (int k = 0; k < 3; k++) {
                Program *p = it.prog[k];
                B.npass[k] = p ? (int)p->sched.n_passes : 0;
                if (p)
                    B.kp[k] = KParams{p->sched.passes, p->sched.rounds, p->sched.ops, p->sched.perms,
                                      p->sched.diags, p->sched.phases, p->sched.term_mo, p->sched.slots,
                                      p->sched.term_q, p->sched.mask_pool, p->sched.cst_mo,
                                      p->sched.cst_q, p->sched.c, p->sched.tw, p->sched.fxt};
                else
                    B.kp[k] = KParams{};
            }
            B.levels = (int64_t)B.npass[0] + (int64_t)B.npass[1] * B.reps_core + B.npass[2];
            max_levels = std::max(max_levels, B.levels);
            for (int64_t j = 0; j < c; j++) cta.push_back((uint16_t)i);
        }
        BatchGroup g{K, smem, (int)cta.size(), max_levels, nullptr, nullptr};
        e.groups.push_back(g);   // freed with the entry if an allocation below fails
        BatchGroup &gg = e.groups.back();
        cudaError_t ce = cudaMalloc((void **)&gg.d_inst, sizeof(BatchInstance) * inst.size());
        if (ce == cudaSuccess) ce = cudaMalloc((void **)&gg.d_cta, sizeof(uint16_t) * cta.size());
        if (ce == cudaSuccess)
            ce = cudaMemcpy(gg.d_inst, inst.data(), sizeof(BatchInstance) * inst.size(), cudaMemcpyHostToDevice);
        if (ce == cudaSuccess)
            ce = cudaMemcpy(gg.d_cta, cta.data(), sizeof(uint16_t) * cta.size(), cudaMemcpyHostToDevice);
        if (ce != cudaSuccess) {
            free_batch(e);
            return fail(ctx, SD_ECUDA, std::string("batch descriptors: ") + cudaGetErrorString(ce));
        }
    }
    // side streams for the instances that run alone, when there is anything
    // to run beside them
    const size_t nside = std::min(kBatchSideStreams, e.alone.size());
    if (nside > 1 || (nside == 1 && !e.groups.empty())) {
        cudaError_t ce = cudaEventCreateWithFlags(&e.fork, cudaEventDisableTiming);
        for (size_t k = 0; k < nside && ce == cudaSuccess; k++) {
            cudaStream_t x = nullptr;
            cudaEvent_t ev = nullptr;
            ce = cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking);
            if (ce == cudaSuccess) e.side.push_back(x);
            if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (ce == cudaSuccess) e.join.push_back(ev);
        }
        if (ce != cudaSuccess) {
            free_batch(e);
            return fail(ctxs[0], SD_ECUDA, std::string("batch streams: ") + cudaGetErrorString(ce));
        }
    }
    g_batches.push_front(std::move(e));
    while (g_batches.size() > kBatchCache) {
        free_batch(g_batches.back());
        g_batches.pop_back();
    }
    out = &g_batches.front();
    return SD_OK;
}

sd_status batch_args(sd_ctx *const *ctxs, void *const *d_states, int64_t count, sd_dtype dtype, double dt,
                     int64_t steps, int order) {
    if (!ctxs || !d_states || count < 0) return fail(nullptr, SD_EINVAL, "invalid batch arguments");
    if (count > 65535) return fail(nullptr, SD_EINVAL, "at most 65535 instances per batch");
    if (steps < 0 || !std::isfinite(dt)) return fail(nullptr, SD_EINVAL, "invalid steps or dt");
    for (int64_t i = 0; i < count; i++) {
        sd_status s = check_state_args(ctxs[i], d_states[i], dtype, order);
        if (s != SD_OK) return s;
    }
    return SD_OK;
}

}  // namespace

extern "C" {

sd_status sd_prepare_batch(sd_ctx *const *ctxs, void *const *d_states, int64_t count, sd_dtype dtype,
                           double dt, int64_t steps, int order) {
    sd_status s = batch_args(ctxs, d_states, count, dtype, dt, steps, order);
    if (s != SD_OK || steps == 0 || count == 0) return s;
    std::lock_guard<std::recursive_mutex> lk(g_batch_mu);
    BatchEntry *e = nullptr;
    return batch_entry(ctxs, d_states, count, dtype, dt, steps, order, nullptr, e);
}

sd_status sd_evolve_batch(sd_ctx *const *ctxs, void *const *d_states, int64_t count, sd_dtype dtype,
                          double dt, int64_t steps, int order, void *cuda_stream) {
    sd_status s = batch_args(ctxs, d_states, count, dtype, dt, steps, order);
    if (s != SD_OK || steps == 0 || count == 0) return s;
    const bool dbl = dtype == SD_C128;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    std::lock_guard<std::recursive_mutex> lk(g_batch_mu);
    BatchEntry *e = nullptr;
    if ((s = batch_entry(ctxs, d_states, count, dtype, dt, steps, order, st, e)) != SD_OK) return s;
    // Instances on the on-chip path, large ones and those with mixed tile
    // sizes run like sd_evolve, side by side on the batch's side streams; the
    // others advance level by level on the caller's stream, one launch per
    // level for each tile size.
    sd_ctx *ctx = ctxs[0];   // where CUDA errors of the fork and join are reported
    if (!e->side.empty()) {
        CK(cudaEventRecord(e->fork, st));
        for (cudaStream_t x : e->side) CK(cudaStreamWaitEvent(x, e->fork, 0));
        for (size_t k = 0; k < e->alone.size(); k++) {
            const int64_t i = e->alone[k];
            if ((s = evolve_impl(ctxs[i], d_states[i], dbl, dt, steps, order, e->side[k % e->side.size()])) != SD_OK)
                return s;
        }
        for (size_t k = 0; k < e->side.size(); k++) CK(cudaEventRecord(e->join[k], e->side[k]));
    } else {
        for (int64_t i : e->alone)
            if ((s = evolve_impl(ctxs[i], d_states[i], dbl, dt, steps, order, st)) != SD_OK) return s;
    }
    for (auto &g : e->groups)
        for (int64_t L = 0; L < g.levels; L++) {
            cudaError_t ce = launch_tile_pass_batch(dbl, g.K, g.d_inst, g.d_cta, g.ctas, g.smem, L, st);
            if (ce != cudaSuccess)
                return fail(ctxs[0], SD_ECUDA, std::string("batch launch: ") + cudaGetErrorString(ce));
        }
    for (cudaEvent_t x : e->join) CK(cudaStreamWaitEvent(st, x, 0));
    return SD_OK;
}

const char *sd_last_error(const sd_ctx *ctx) {
    if (ctx && !ctx->err.empty()) return ctx->err.c_str();
    return g_last_error.c_str();
}

void sd_destroy(sd_ctx *ctx) { delete ctx; }

}  // extern "C"
