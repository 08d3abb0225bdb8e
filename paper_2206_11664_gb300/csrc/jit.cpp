// Run-time specialisation of tile passes.
//
// The interpreter kernel (kernels.cu) reads each pass's rounds and ops from
// device memory and dispatches on them; for large states that dispatch and
// the register traffic it forces dominate a pass.  Here every pass of a
// schedule becomes straight-line CUDA C++ -- layouts, register slots,
// Clifford phases, class boundaries, global offsets and scales as
// constants -- compiled once with NVRTC for sm_103a and launched through the
// driver API.  The generated kernels compute what the interpreter computes,
// op for op, with the same device helpers (tile_device.cuh).
#include <cuda.h>
#include <cuda_runtime.h>
#include <dlfcn.h>
#include <nvrtc.h>
#include <sys/stat.h>
#include <unistd.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <functional>
#include <map>
#include <mutex>
#include <atomic>
#include <thread>
#include <algorithm>
#include <cmath>
#include <sstream>
#include <string>
#include <vector>

#include "jit.h"
#include "jit_headers.inc"   // kJitDevTypes, kJitFixedPoint, kJitTileDevice: the device headers as text

namespace sd {
namespace {

struct Nvrtc {
    bool ok = false;
    nvrtcResult (*create)(nvrtcProgram *, const char *, const char *, int, const char *const *,
                          const char *const *) = nullptr;
    nvrtcResult (*compile)(nvrtcProgram, int, const char *const *) = nullptr;
    nvrtcResult (*log_size)(nvrtcProgram, size_t *) = nullptr;
    nvrtcResult (*log)(nvrtcProgram, char *) = nullptr;
    nvrtcResult (*cubin_size)(nvrtcProgram, size_t *) = nullptr;
    nvrtcResult (*cubin)(nvrtcProgram, char *) = nullptr;
    nvrtcResult (*destroy)(nvrtcProgram *) = nullptr;
    nvrtcResult (*version)(int *, int *) = nullptr;
};

struct Driver {
    bool ok = false;
    CUresult (*load)(CUmodule *, const void *) = nullptr;
    CUresult (*get_function)(CUfunction *, CUmodule, const char *) = nullptr;
    CUresult (*set_attr)(CUfunction, CUfunction_attribute, int) = nullptr;
    CUresult (*launch)(CUfunction, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned,
                       unsigned, CUstream, void **, void **) = nullptr;
    CUresult (*occupancy)(int *, CUfunction, int, size_t) = nullptr;
};

std::mutex g_mu;
Nvrtc g_nvrtc;
Driver g_drv;
bool g_init = false;
std::string g_why;
std::map<std::string, CUmodule> g_modules;   // source hash -> loaded module

template <typename F>
bool sym(void *h, const char *name, F &f) {
    f = reinterpret_cast<F>(dlsym(h, name));
    return f != nullptr;
}

template <typename F>
bool drv_sym(const char *name, F &f) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p) {
        cudaGetLastError();
        return false;
    }
    f = reinterpret_cast<F>(p);
    return true;
}

void init_locked() {
    if (g_init) return;
    g_init = true;
    const char *cands[] = {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13",
                           "/usr/local/cuda/lib64/libnvrtc.so"};
    void *h = nullptr;
    for (const char *c : cands)
        if ((h = dlopen(c, RTLD_NOW | RTLD_LOCAL))) break;
    if (!h) {
        g_why = "libnvrtc not found";
        return;
    }
    g_nvrtc.ok = sym(h, "nvrtcCreateProgram", g_nvrtc.create) &&
                 sym(h, "nvrtcCompileProgram", g_nvrtc.compile) &&
                 sym(h, "nvrtcGetProgramLogSize", g_nvrtc.log_size) &&
                 sym(h, "nvrtcGetProgramLog", g_nvrtc.log) &&
                 sym(h, "nvrtcGetCUBINSize", g_nvrtc.cubin_size) &&
                 sym(h, "nvrtcGetCUBIN", g_nvrtc.cubin) &&
                 sym(h, "nvrtcDestroyProgram", g_nvrtc.destroy) &&
                 sym(h, "nvrtcVersion", g_nvrtc.version);
    if (!g_nvrtc.ok) {
        g_why = "libnvrtc lacks a needed symbol";
        return;
    }
    g_drv.ok = drv_sym("cuModuleLoadData", g_drv.load) &&
               drv_sym("cuModuleGetFunction", g_drv.get_function) &&
               drv_sym("cuFuncSetAttribute", g_drv.set_attr) &&
               drv_sym("cuLaunchKernel", g_drv.launch) &&
               drv_sym("cuOccupancyMaxActiveBlocksPerMultiprocessor", g_drv.occupancy);
    if (!g_drv.ok) g_why = "CUDA driver entry points unavailable";
}

// ------------------------------------------------------------ code generation

std::string hex64(uint64_t v) {
    char b[40];
    snprintf(b, sizeof b, "0x%llxull", (unsigned long long)v);
    return b;
}
std::string hex32(uint32_t v) {
    char b[24];
    snprintf(b, sizeof b, "0x%xu", v);
    return b;
}
std::string dbl(double v) {
    char b[48];
    snprintf(b, sizeof b, "%.17g", v);
    return b;
}

// XOR of col(p) over the tile positions p that the thread's lane and warp
// bits select in round R (32-bit or 64-bit result).
std::string thread_expr(const DevRound &R, int K, const std::function<uint64_t(int)> &col, bool wide) {
    std::ostringstream o;
    o << (wide ? "(0ull" : "(0u");
    for (int i = 0; i < kLaneBits; i++) {
        uint64_t v = col(R.lane_pos[i]);
        if (v) o << " ^ ((" << (wide ? "uint64_t" : "uint32_t") << ")((lane >> " << i << ") & 1) * "
                 << (wide ? hex64(v) : hex32((uint32_t)v)) << ")";
    }
    for (int i = 0; i < K - 9; i++) {
        uint64_t v = col(R.warp_pos[i]);
        if (v) o << " ^ ((" << (wide ? "uint64_t" : "uint32_t") << ")((warp >> " << i << ") & 1) * "
                 << (wide ? hex64(v) : hex32((uint32_t)v)) << ")";
    }
    o << ")";
    return o.str();
}

// Generated kernel of pass pi: sd_pass_c64_<pi> or sd_pass_c128_<pi>.
std::string kernel_name(int pi, bool dbl_state) {
    return std::string(dbl_state ? "sd_pass_c128_" : "sd_pass_c64_") + std::to_string(pi);
}

// Fixed-point one-qubit Cliffords on register slot I.  Register s holds its
// amplitude times i^-kph[s] (kph fixed at generation time, since the slot
// bits are): the output phase i^B of S^B H S^PA stays in kph, and i^m for the
// operands' phase difference m only chooses adds or subtracts of the parts.
void emit_had_fx(std::ostringstream &o, int I, int PA, int B, int *kph) {
    static const char *form[4] = {
        "ar[%d] = ur + vr; ai[%d] = ui + vi; ar[%d] = ur - vr; ai[%d] = ui - vi;",
        "ar[%d] = ur - vi; ai[%d] = ui + vr; ar[%d] = ur + vi; ai[%d] = ui - vr;",
        "ar[%d] = ur - vr; ai[%d] = ui - vi; ar[%d] = ur + vr; ai[%d] = ui + vi;",
        "ar[%d] = ur + vi; ai[%d] = ui - vr; ar[%d] = ur - vi; ai[%d] = ui + vr;"};
    for (int s = 0; s < 16; s++) {
        if ((s >> I) & 1) continue;
        const int t = s | (1 << I);
        const int m = (PA + kph[t] - kph[s]) & 3;
        char buf[256];
        snprintf(buf, sizeof buf, form[m], s, s, t, t);
        o << "      { const long long ur = ar[" << s << "], ui = ai[" << s << "], vr = ar[" << t << "], vi = ai[" << t
          << "]; " << buf << " }\n";
        kph[t] = (B + kph[s]) & 3;
    }
}
void emit_mono_fx(std::ostringstream &o, int I, int PA, int XX, int *kph) {
    for (int s = 0; s < 16; s++) {
        if ((s >> I) & 1) continue;
        const int t = s | (1 << I);
        kph[t] = (kph[t] + PA) & 3;
        if (XX) {
            o << "      { const long long r = ar[" << s << "], i = ai[" << s << "]; ar[" << s << "] = ar[" << t
              << "]; ai[" << s << "] = ai[" << t << "]; ar[" << t << "] = r; ai[" << t << "] = i; }\n";
            std::swap(kph[s], kph[t]);
        }
    }
}

// ---------------------------------------------------- complex64 butterflies
// A complex64 register slot may hold its amplitude v in one of eight
// representations fixed at generation time: the stored pair p has
// re v = sr p[sw] and im v = si p[1 - sw].  A butterfly (u, v) -> (u + i^PA v,
// i^B (u - i^PA v)) whose two operands are stored with the same sw (after the
// i^PA) is two packed f32x2 operations, u + D w and u - D w with a sign pair
// D, and its second output simply takes the first operand's representation
// times i^B.  Otherwise it is four scalar adds (signs and order are free in
// scalar code), whose outputs may take any representation: the generator
// picks those, and the output representations of a group exponential's
// rotation, so that the following butterflies of the round pack.  Every slot
// returns to the plain representation (sw = 0, sr = si = 1) before a store,
// a quarter-turn layer and the end of the round.
struct SlotRep {
    int sw = 0, sr = 1, si = 1;
};

bool rep_plain(const SlotRep &r) { return r.sw == 0 && r.sr == 1 && r.si == 1; }

// the representation of i^k v, stored in the same pair as v
SlotRep rep_mul_i(SlotRep r, int k) {
    for (k &= 3; k > 0; k--) r = SlotRep{1 - r.sw, -r.si, r.sr};
    return r;
}

// A true component as a signed stored component: sign and index (0: .x, 1: .y).
struct Comp {
    int sign, idx;
};
Comp comp_re(const SlotRep &r) { return Comp{r.sr, r.sw}; }
Comp comp_im(const SlotRep &r) { return Comp{r.si, 1 - r.sw}; }

// sa a + sb b as one add with operand signs
std::string signed_sum(int sa, const std::string &a, int sb, const std::string &b) {
    if (sa > 0) return a + (sb > 0 ? " + " : " - ") + b;
    if (sb > 0) return b + " - " + a;
    return "-" + a + " - " + b;
}

struct C64Rounds {
    SlotRep rep[16];

    void reset() {
        for (auto &r : rep) r = SlotRep{};
    }
    // instructions that bring the slots rp back to the plain representation
    static int fixup_cost(const SlotRep *rp) {
        int c = 0;
        for (int s = 0; s < 16; s++) c += rep_plain(rp[s]) ? 0 : (rp[s].sw ? 2 : 1);
        return c;
    }
    static bool packable(const SlotRep *rp, int I, int PA) {
        for (int s = 0; s < 16; s++) {
            if ((s >> I) & 1) continue;
            if (rp[s].sw != rep_mul_i(rp[s | (1 << I)], PA).sw) return false;
        }
        return true;
    }
    // Representations that a scalar butterfly or a rotation at op k leaves:
    // sw = parity of (s & L), signs +, for the L whose representations let
    // the most following butterflies of the round pack.
    static void target(const Schedule &S, const DevRound &R, int k, SlotRep *out) {
        int best_L = 0, best = -1;
        for (int L = 0; L < 16; L++) {
            SlotRep rp[16];
            for (int s = 0; s < 16; s++) rp[s] = SlotRep{__builtin_popcount(s & L) & 1, 1, 1};
            int packed = 0;
            for (int oi = k + 1; oi < R.op_end; oi++) {
                const DevOp &op = S.ops[oi];
                if (op.kind == D_PHASE || op.kind == D_DIAG) break;
                const int I = op.slot;
                if (op.kind == D_MONO) {
                    for (int s = 0; s < 16; s++) {
                        if ((s >> I) & 1) continue;
                        const int t = s | (1 << I);
                        rp[t] = rep_mul_i(rp[t], c1_a(op.arg));
                        if (c1_x(op.arg)) std::swap(rp[s], rp[t]);
                    }
                    continue;
                }
                if (!packable(rp, I, c1_a(op.arg))) break;
                packed++;
                for (int s = 0; s < 16; s++)
                    if (!((s >> I) & 1)) rp[s | (1 << I)] = rep_mul_i(rp[s], c1_b(op.arg));
            }
            if (packed > best || (packed == best && __builtin_popcount(L) < __builtin_popcount(best_L))) {
                best = packed;
                best_L = L;
            }
        }
        for (int s = 0; s < 16; s++) out[s] = SlotRep{__builtin_popcount(s & best_L) & 1, 1, 1};
    }
    // whether op k is the round's last butterfly or rotation before the next
    // quarter-turn layer or the round's end
    static bool last_before_plain(const Schedule &S, const DevRound &R, int k) {
        for (int oi = k + 1; oi < R.op_end; oi++) {
            const int kind = S.ops[oi].kind;
            if (kind == D_PHASE) return true;
            if (kind == D_HAD || kind == D_DIAG) return false;
        }
        return true;
    }
    // reps after the ops k+1.. up to the next quarter-turn layer (monos only
    // when op k is the last butterfly)
    void after_monos(const Schedule &S, const DevRound &R, int k, SlotRep *rp) const {
        for (int oi = k + 1; oi < R.op_end; oi++) {
            const DevOp &op = S.ops[oi];
            if (op.kind != D_MONO) break;
            for (int s = 0; s < 16; s++) {
                if ((s >> op.slot) & 1) continue;
                const int t = s | (1 << op.slot);
                rp[t] = rep_mul_i(rp[t], c1_a(op.arg));
                if (c1_x(op.arg)) std::swap(rp[s], rp[t]);
            }
        }
    }

    void had(std::ostringstream &o, const Schedule &S, const DevRound &R, int k, bool free_fixup) {
        const DevOp &op = S.ops[k];
        const int I = op.slot, PA = c1_a(op.arg), B = c1_b(op.arg);
        bool pack = packable(rep, I, PA);
        const bool last = last_before_plain(S, R, k);
        for (int oi = k + 1; oi < R.op_end; oi++)   // a quarter-turn layer comes before the store
            if (S.ops[oi].kind == D_PHASE) free_fixup = false;
        SlotRep out[16];
        if (pack && last && !free_fixup) {
            // packed, then back to plain, against scalar with plain outputs
            SlotRep rp[16];
            for (int s = 0; s < 16; s++) rp[s] = rep[s];
            for (int s = 0; s < 16; s++)
                if (!((s >> I) & 1)) rp[s | (1 << I)] = rep_mul_i(rp[s], B);
            after_monos(S, R, k, rp);
            pack = 16 + fixup_cost(rp) <= 32;
        }
        if (!pack) {
            if (last) {
                for (auto &r : out) r = SlotRep{};
            } else {
                target(S, R, k, out);
            }
        }
        for (int s = 0; s < 16; s++) {
            if ((s >> I) & 1) continue;
            const int t = s | (1 << I);
            const SlotRep Rs = rep[s], Rw = rep_mul_i(rep[t], PA);
            if (pack) {
                float d[2];
                d[Rs.sw] = (float)(Rs.sr * Rw.sr);
                d[1 - Rs.sw] = (float)(Rs.si * Rw.si);
                auto add = [&](float e0, float e1) -> std::string {
                    if (e0 > 0 && e1 > 0) return "__fadd2_rn(u, v)";
                    return std::string("__ffma2_rn(v, make_float2(") + (e0 > 0 ? "1.f" : "-1.f") + ", " +
                           (e1 > 0 ? "1.f" : "-1.f") + "), u)";
                };
                o << "      { const A u = a[" << s << "], v = a[" << t << "]; a[" << s << "] = " << add(d[0], d[1])
                  << "; a[" << t << "] = " << add(-d[0], -d[1]) << "; }\n";
                rep[t] = rep_mul_i(Rs, B);
            } else {
                // true parts of u, w = i^PA v and the outputs, as signed stored parts
                static const char *sn[2] = {"s0", "s1"}, *tn[2] = {"t0", "t1"};
                const Comp ur = comp_re(Rs), ui = comp_im(Rs), wr = comp_re(Rw), wi = comp_im(Rw);
                // out1 = u + w; dif = u - w; out2 = i^B dif
                struct Sum {
                    int sa, ia, sb, ib;   // sa s[ia] + sb t[ib]
                };
                Sum o1r{ur.sign, ur.idx, wr.sign, wr.idx}, o1i{ui.sign, ui.idx, wi.sign, wi.idx};
                Sum dr{ur.sign, ur.idx, -wr.sign, wr.idx}, di{ui.sign, ui.idx, -wi.sign, wi.idx};
                for (int b = 0; b < (B & 3); b++) {   // i (re + i im) = -im + i re
                    const Sum nr{-di.sa, di.ia, -di.sb, di.ib};
                    di = dr;
                    dr = nr;
                }
                auto store = [&](int slot, const SlotRep &ro, const Sum &re, const Sum &im) {
                    // p[sw] = sr re, p[1 - sw] = si im
                    const Sum c0 = ro.sw ? im : re, c1 = ro.sw ? re : im;
                    const int f0 = ro.sw ? ro.si : ro.sr, f1 = ro.sw ? ro.sr : ro.si;
                    o << " a[" << slot << "].x = " << signed_sum(f0 * c0.sa, sn[c0.ia], f0 * c0.sb, tn[c0.ib])
                      << "; a[" << slot << "].y = " << signed_sum(f1 * c1.sa, sn[c1.ia], f1 * c1.sb, tn[c1.ib])
                      << ";";
                };
                o << "      { const float s0 = a[" << s << "].x, s1 = a[" << s << "].y, t0 = a[" << t
                  << "].x, t1 = a[" << t << "].y;";
                store(s, out[s], o1r, o1i);
                store(t, out[t], dr, di);
                o << " }\n";
            }
        }
        if (!pack)
            for (int s = 0; s < 16; s++) rep[s] = out[s];
    }

    void mono(std::ostringstream &o, const DevOp &op) {
        const int I = op.slot;
        for (int s = 0; s < 16; s++) {
            if ((s >> I) & 1) continue;
            const int t = s | (1 << I);
            rep[t] = rep_mul_i(rep[t], c1_a(op.arg));
            if (c1_x(op.arg)) {
                o << "      { const A w = a[" << s << "]; a[" << s << "] = a[" << t << "]; a[" << t << "] = w; }\n";
                std::swap(rep[s], rep[t]);
            }
        }
    }

    // back to the plain representation
    void plain(std::ostringstream &o) {
        for (int s = 0; s < 16; s++) {
            const SlotRep r = rep[s];
            if (rep_plain(r)) continue;
            if (r.sw == 0)
                o << "      a[" << s << "] = __fmul2_rn(a[" << s << "], make_float2(" << (r.sr > 0 ? "1.f" : "-1.f")
                  << ", " << (r.si > 0 ? "1.f" : "-1.f") << "));\n";
            else
                o << "      a[" << s << "] = make_float2(" << (r.sr > 0 ? "" : "-") << "a[" << s << "].y, "
                  << (r.si > 0 ? "" : "-") << "a[" << s << "].x);\n";
            rep[s] = SlotRep{};
        }
    }

    // The group exponential's rotation of every slot, from its current
    // representation to the ones the following butterflies want.
    void rotate(std::ostringstream &o, const Schedule &S, const DevRound &R, int k, double sc) {
        SlotRep out[16];
        if (last_before_plain(S, R, k)) {
            for (auto &r : out) r = SlotRep{};
        } else {
            target(S, R, k, out);
        }
        o << "        { uint32_t g[16];\n"
          << "          #pragma unroll\n"
          << "          for (int s = 0; s < 16; s++) g[s] = (uint32_t)(G[s] >> 32);\n"
          << "          wht16(g);\n";
        for (int s = 0; s < 16; s++) {
            const SlotRep &ri = rep[s], &ro = out[s];
            o << "          a[" << s << "] = rotate_tw32_rep<" << ri.sw << ", " << ri.sr << ", " << ri.si << ", "
              << ro.sw << ", " << ro.sr << ", " << ro.si << ">(a[" << s << "], g[" << s << "], TW, (T)" << dbl(sc)
              << ");\n";
        }
        o << "        }\n";
        for (int s = 0; s < 16; s++) rep[s] = out[s];
    }
};

// Limits of the straight-line code emitted for a round's group exponentials.
constexpr int kInlineTerms = 384;   // terms staged per round
constexpr int kInlineSlots = 192;   // slots per round / per exponential

// Whether class u of a group exponential has any term on the tile.
bool diag_class_used(const DevDiag &d, int u) {
    return d.off[u + 1] > d.off[u] || d.zs[u] >= 0 || (u == 0 && d.cst >= 0);
}

// Whether a round's staging is emitted as straight-line code (rounds of
// modest size: longer code compiles slowly and gains nothing once the work is
// spread out).
bool round_inline_stage(const Schedule &S, const DevRound &R) {
    int round_terms = 0;
    for (int j = 0; j < R.slot_count; j++) round_terms += S.slots[R.slot_begin + j].tn;
    return round_terms <= kInlineTerms && R.slot_count <= kInlineSlots;
}

// The slot sums of a round's group exponentials for the tile (into ST) and
// its tile-constant sums (into CST), without barriers.
void emit_slot_sums(std::ostringstream &o, const Schedule &S, const DevPass &P, const DevRound &R, int NT) {
    const bool inline_stage = round_inline_stage(S, R);
    if (P.term_cache && !inline_stage) {
        o << "      stage_slots(xo, kp.slots, " << R.slot_begin << ", " << R.slot_count
          << ", TCM, TCQ, " << P.term_begin << ", ST, tid, NT);\n";
    } else if (P.term_cache) {
        // one thread per slot, spread over the warps; masks inline, angles from the cache
        for (int j = 0; j < R.slot_count; j++) {
            const DevSlot &sl = S.slots[R.slot_begin + j];
            const int thr = ((j * 32) % NT + (j * 32) / NT) % NT;
            o << "      if (tid == " << thr << ") { uint64_t acc = 0ull;\n";
            for (int t = sl.tb; t < sl.tb + sl.tn; t++) {
                const int i = t - P.term_begin;
                o << "        { const uint64_t v = (uint64_t)TCQ[" << i << "]; acc += (__popcll(xo & "
                  << hex64(S.term_mo[t]) << ") & 1) ? 0ull - v : v; }\n";
            }
            o << "        ST[" << j << "].q = acc; ST[" << j << "].ml = " << hex32(sl.ml) << "; }\n";
        }
    } else {
        o << "      stage_slots(xo, kp.slots, " << R.slot_begin << ", " << R.slot_count
          << ", kp.term_mo, kp.term_q, 0, ST, tid, NT);\n";
    }
    for (int cc = 0; cc < 4; cc++)
        if (R.cst_count[cc] > 0)
            o << "      if (warp == " << (cc % (NT / 32)) << ") { const uint64_t v = warp_const_sum(xo, kp.cst_mo, kp.cst_q, "
              << R.cst_begin[cc] << ", " << R.cst_count[cc] << ", lane); if (lane == 0) CST[" << cc << "] = v; }\n";
}

// Staging of a round's group exponentials for the tile (slot sums, tile
// constants, class totals), with the barriers around it.  Complex64 passes
// bias the class totals by 2^31 (rounding to Q0.32 turns), complex128 passes
// keep Q0.64.
void emit_round_staging(std::ostringstream &o, const Schedule &S, const DevPass &P, const DevRound &R, int NT,
                        bool dbl_state) {
    const bool inline_stage = round_inline_stage(S, R);
    emit_slot_sums(o, S, P, R, NT);
    o << "      __syncthreads();\n";
    // class totals, one thread each, spread over the warps
    if (!inline_stage)
        o << "      stage_totals(kp, " << R.diag_begin << ", " << R.n_diag << ", ST, CST, "
          << hex64(dbl_state ? 0 : (1ull << 31)) << ", TQ, tid, NT);\n";
    for (int k = 0; k < R.n_diag && inline_stage; k++) {
        const DevDiag &d = S.diags[R.diag_begin + k];
        for (int u = 0; u < 16; u++) {
            if (!diag_class_used(d, u)) continue;
            const int i = d.tot + u;
            const int thr = ((i * 32) % NT + (i * 32) / NT) % NT;
            o << "      if (tid == " << thr << ") TQ[" << i << "] = " << hex64(dbl_state ? 0 : (1ull << 31));
            if (d.zs[u] >= 0) o << " + ST[" << d.zs[u] << "].q";
            for (int j = d.off[u]; j < d.off[u + 1]; j++) o << " + ST[" << j << "].q";
            if (u == 0 && d.cst >= 0) o << " + CST[" << d.cst << "]";
            o << ";\n";
        }
    }
    o << "      __syncthreads();\n";
}

// The round of a pass whose staging moves into the round before it: the
// pass's only round with group exponentials, if its staging is straight-line
// code.  Its slot sums are then formed while the previous round runs (for
// the first round: in the last round of the previous tile, and before the
// loop for the block's first tile), the barrier that opens the round orders
// them, and each thread forms its class totals itself (emit_class_sums_full),
// so that the round needs no barriers of its own for the staging.  A pass of
// one round keeps its staging in place.  -1 if none.
int hoisted_stage_round(const Schedule &S, const DevPass &P) {
    int found = -1, count = 0;
    for (int r = 0; r < P.n_rounds; r++)
        if (S.rounds[P.round_begin + r].n_diag > 0) {
            found = r;
            count++;
        }
    if (count != 1 || P.n_rounds < 2) return -1;
    return round_inline_stage(S, S.rounds[P.round_begin + found]) ? found : -1;
}

// The round in which the hoisted staging of round h is emitted: the round
// before it, or the pass's last round (for the next tile) when h = 0.
int staging_round(const DevPass &P, int h) { return h > 0 ? h - 1 : P.n_rounds - 1; }

// Slot sums of the hoisted round h, emitted in round r = staging_round(h):
// for this tile, or (h = 0) for the block's next tile.
void emit_hoisted_slot_sums(std::ostringstream &o, const Schedule &S, const DevPass &P, int h, int NT) {
    const DevRound &H = S.rounds[P.round_begin + h];
    if (h > 0) {
        emit_slot_sums(o, S, P, H, NT);
        return;
    }
    o << "      if (tile + gridDim.x < ntiles) {\n        const uint64_t xo = deposit(tile + gridDim.x);\n";
    emit_slot_sums(o, S, P, H, NT);
    o << "      }\n";
}

// Whether round r (r >= 1) of a pass may open with a warp barrier instead of
// a block barrier: it holds the same tile positions on the warp index as
// round r - 1 (so every amplitude a warp reads from the exchange was written
// by that warp), round r - 1 wrote the exchange without a permutation, and
// round r reads nothing that other warps staged (its own staging, or the
// slot sums hoisted into round r - 1).
bool warp_local_round(const Schedule &S, const DevPass &P, int r, int hoist) {
    if (r < 1) return false;
    const DevRound &A = S.rounds[P.round_begin + r - 1], &B = S.rounds[P.round_begin + r];
    if (A.perm >= 0 || B.n_diag > 0 || r == hoist) return false;
    if (hoist >= 0 && staging_round(P, hoist) == r - 1) return false;
    const int nw = S.K - kRegBits - kLaneBits;
    uint32_t wa = 0, wb = 0;
    for (int i = 0; i < nw; i++) {
        wa |= 1u << A.warp_pos[i];
        wb |= 1u << B.warp_pos[i];
    }
    return wa == wb;
}

// The round after whose opening block barrier a pass with one prefetch
// buffer issues the next tile's prefetch: the first round r >= 1 that opens
// with a block barrier (every thread has read the buffer in round 0 by then).
// 0 when there is none: the prefetch then follows a barrier of its own in
// round 0.
int prefetch_round(const Schedule &S, const DevPass &P, int hoist) {
    for (int r = 1; r < P.n_rounds; r++)
        if (!warp_local_round(S, P, r, hoist)) return r;
    return 0;
}

// Dynamic shared memory of a generated pass: the interpreter's layout
// (exchange buffer, prefetch buffer, staging, term cache) plus, when asked
// for and when it fits, a second prefetch buffer, so that two tiles are in
// flight while the block works on a third.
size_t jit_pass_smem(const Schedule &S, const DevPass &P, size_t amp, int K, bool *two) {
    const size_t base = pass_smem_bytes(P, amp, K);
    // prefetch 3: two buffers in the passes without a group exponential only
    const bool want = S.prefetch == 2 || (S.prefetch == 3 && !P.scale_in_diag);
    const bool t = want && base + (amp << K) <= kTileSmemLimit;
    if (two) *two = t;
    return t ? base + (amp << K) : base;
}

// Class sums G[u] of a group exponential formed by the thread from the
// staged slots alone: the bias, the class's slot constant over the fixed
// positions, the tile constant (class 0), and each other slot of the class
// with the sign of its parity with lf.
void emit_class_sums_full(std::ostringstream &o, const Schedule &S, const DevRound &R, const DevDiag &d,
                          uint64_t bias) {
    for (int u = 0; u < 16; u++) {
        if (!diag_class_used(d, u)) {
            o << "        G[" << u << "] = 0ull;\n";
            continue;
        }
        o << "        { uint64_t o0 = " << hex64(bias) << ", o1 = 0ull;\n";
        if (d.zs[u] >= 0) o << "          o1 += ST[" << d.zs[u] << "].q;\n";
        if (u == 0 && d.cst >= 0) o << "          o1 += CST[" << d.cst << "];\n";
        for (int j = d.off[u]; j < d.off[u + 1]; j++) {
            const uint32_t ml = S.slots[R.slot_begin + j].ml;
            const char *acc = ((j - d.off[u]) & 1) ? "o1" : "o0";
            o << "          { const uint64_t q = ST[" << j << "].q; " << acc << " += ";
            if ((ml & (ml - 1)) == 0) o << "(lf & " << hex32(ml) << ")";
            else o << "(__popc(lf & " << hex32(ml) << ") & 1)";
            o << " ? 0ull - q : q; }\n";
        }
        o << "          G[" << u << "] = o0 + o1; }\n";
    }
}

// Class sums G[u] of a group exponential for the thread (fixed positions lf):
// the class total less twice its slots of odd parity with lf.
void emit_class_sums(std::ostringstream &o, const Schedule &S, const DevRound &R, const DevDiag &d) {
    const bool unrolled = d.off[16] <= kInlineSlots;
    for (int u = 0; u < 16; u++) {
        if (!diag_class_used(d, u)) {
            o << "        G[" << u << "] = 0ull;\n";
            continue;
        }
        const int b = d.off[u], e = d.off[u + 1];
        o << "        { uint64_t o0 = 0ull, o1 = 0ull;\n";
        if (unrolled) {
            for (int j = b; j < e; j++) {
                const uint32_t ml = S.slots[R.slot_begin + j].ml;
                const char *acc = ((j - b) & 1) ? "o1" : "o0";
                if ((ml & (ml - 1)) == 0)
                    o << "          if (lf & " << hex32(ml) << ") " << acc << " += ST[" << j << "].q;\n";
                else
                    o << "          if (__popc(lf & " << hex32(ml) << ") & 1) " << acc << " += ST[" << j
                      << "].q;\n";
            }
        } else if (e > b) {
            o << "          #pragma unroll 4\n"
              << "          for (int j = " << b << "; j < " << e << "; j++) {\n"
              << "            const StagedTerm t0 = ST[j];\n"
              << "            if (__popc(lf & t0.ml) & 1) o0 += t0.q;\n"
              << "          }\n";
        }
        o << "          G[" << u << "] = TQ[" << d.tot + u << "] - 2ull * (o0 + o1); }\n";
    }
}

// The tile bookkeeping every pass kernel opens with: the thread's share of
// the prefetch copy, the tile count, the outer-bit deposit of a tile index
// and the cp.async prefetch of a tile into Pf (natural tile order, E
// amplitudes per 16-byte copy).
void emit_io_prologue(std::ostringstream &o, const DevPass &P, int K, int NT, int E, int n) {
    auto gbit = [&](int p) -> uint64_t { return (uint64_t)1 << P.tile_bits[p]; };
    const int NCOPY = (1 << K) / E / NT;
    // copy l = (tid + k NT) E: bit j of l is bit (j - log2 E) of tid for the low K-4 such bits
    const int le = E == 2 ? 1 : 0;
    o << "  const uint64_t sp_tid = 0ull";
    for (int j = le; j < K; j++)
        if (j - le < K - 4) o << " | ((uint64_t)((tid >> " << (j - le) << ") & 1) << " << (int)P.tile_bits[j] << ")";
    o << ";\n  const long long ntiles = " << (1LL << (n - K)) << "ll;\n"
      << "  auto deposit = [&](long long t) -> uint64_t {\n"
      << "    return OUTT[0][t & 255] | OUTT[1][(t >> 8) & 255] | OUTT[2][(t >> 16) & 255] | OUTT[3][(t >> 24) & 255];\n"
      << "  };\n"
      << "  auto prefetch = [&](long long t, A *buf) {\n    const uint64_t xo = deposit(t) | sp_tid;\n";
    for (int k = 0; k < NCOPY; k++) {
        const uint64_t lk = (uint64_t)k * NT * E;
        uint64_t off = 0;
        for (int j = 0; j < K; j++)
            if ((lk >> j) & 1) off |= gbit(j);
        o << "    cp_async16(buf + (tid * E + " << lk << "), psi + (xo | " << hex64(off) << "));\n";
    }
    o << "    cp_async_commit();\n  };\n";
}

std::string gen_pass(const Schedule &S, int pi, int n, bool dbl_state) {
    const DevPass &P = S.passes[pi];
    const int K = S.K, c = S.c;
    const int NT = 1 << (K - 4);
    const int E = dbl_state ? 1 : 2;
    auto gbit = [&](int p) -> uint64_t { return (uint64_t)1 << P.tile_bits[p]; };
    auto swc = [&](int p) -> uint64_t { return swizzle_col(p, c); };
    auto lcol = [&](int p) -> uint64_t { return (uint64_t)1 << p; };
    const double pass_scale = P.scale_in_diag ? 1.0 : P.scale;
    // With a single group exponential in the pass, the pass scale goes into
    // the rotation table instead of two multiplies per amplitude.
    int n_diag = 0;
    for (int r = 0; r < P.n_rounds; r++) {
        const DevRound &R = S.rounds[P.round_begin + r];
        for (int oi = R.op_begin; oi < R.op_end; oi++) n_diag += S.ops[oi].kind == D_DIAG;
    }
    const bool table_scaled = P.scale_in_diag && n_diag == 1;
    const double table_scale = table_scaled ? P.scale : 1.0;
    const int hoist = hoisted_stage_round(S, P);
    bool two = false;
    jit_pass_smem(S, P, dbl_state ? 16 : 8, K, &two);
    // With two prefetch buffers the next two tiles are in flight: tile t's
    // buffer, once every thread has read it, receives tile t + 2 grid.
    const std::string pf_next = two ? "      if (tile + 2ll * gridDim.x < ntiles) prefetch(tile + 2ll * gridDim.x, Pf);\n"
                                    : "      if (tile + gridDim.x < ntiles) prefetch(tile + gridDim.x, Pf);\n";
    const int pf_round = prefetch_round(S, P, hoist);
    // Complex128 passes run in fixed point (fx): each round ends with an
    // arithmetic shift that applies the 1/2 of each pair of its Hadamards
    // (a lone 1/sqrt(2) is carried to the next round); one left at the end of
    // the pass goes into the rotation table of its only group exponential,
    // or (none or several of them) into a multiply before the
    // store.  Headroom fx_hr: a tile's norm is invariant in a pass, so a
    // component never exceeds 2^((K+1)/2) times the tile's largest one, and a
    // round's unnormalised butterflies add at most (h+1)/2 bits before its shift.
    const bool fx = dbl_state;
    std::vector<int> fx_shift(P.n_rounds, 0);
    int fx_hmax = 0, fx_pend = 0;
    for (int r = 0; r < P.n_rounds; r++) {
        const DevRound &R = S.rounds[P.round_begin + r];
        int h = 0;
        for (int oi = R.op_begin; oi < R.op_end; oi++) h += S.ops[oi].kind == D_HAD;
        fx_hmax = std::max(fx_hmax, h);
        fx_shift[r] = (fx_pend + h) >> 1;
        fx_pend = (fx_pend + h) & 1;
    }
    const int fx_hr = (K + 2) / 2 + 2 + (fx_hmax + 2) / 2;
    const bool fx_res_table = fx && fx_pend && n_diag == 1;
    const bool fx_res_store = fx && fx_pend && n_diag != 1;
    std::ostringstream o;
    o << "extern \"C\" __global__ void __launch_bounds__(" << NT << ") " << kernel_name(pi, dbl_state)
      << "(A *__restrict__ psi, sd::KParams kp) {\n"
      << "  using namespace sd;\n"
      << "  constexpr int K = " << K << ", NT = " << NT << ", E = " << E << ";\n"
      << "  extern __shared__ __align__(16) unsigned char smraw[];\n"
      << "  A *X = reinterpret_cast<A *>(smraw);\n"
      << "  A *Pf0 = X + (1 << K), *Pf1 = Pf0 + " << (two ? "(1 << K)" : "0") << ";\n"
      << "  StagedTerm *ST = reinterpret_cast<StagedTerm *>(Pf0 + " << (two ? 2 : 1) << " * (1 << K));\n"
      << "  uint64_t *TQ = reinterpret_cast<uint64_t *>(ST + " << (P.max_stage > 0 ? P.max_stage : 1) << ");\n"
      << "  (void)ST; (void)TQ;\n";
    if (P.term_cache)
        o << "  uint64_t *TCM = TQ + " << P.max_tot << ";\n"
          << "  int64_t *TCQ = reinterpret_cast<int64_t *>(TCM + " << P.term_count << ");\n"
          << "  cache_terms(kp, " << P.term_begin << ", " << P.term_count << ", TCM, TCQ, threadIdx.x, NT);\n";
    if (fx)
        o << "  longlong2 *XI = reinterpret_cast<longlong2 *>(X);\n"
          << "  __shared__ longlong2 T1[256], T2[256];\n"
          << "  __shared__ uint32_t EM[NT / 32];\n";
    else
        o << "  __shared__ A TW[256];\n";
    o
      << "  __shared__ uint64_t OUTT[4][256];\n"
      << "  __shared__ uint64_t CST[4];\n"
      << "  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;\n"
      << "  (void)lane; (void)warp;\n"
      << "  for (int i = tid; i < 256; i += NT) {\n";
    if (fx) {
        if (fx_res_table)   // the pass's remaining 1/sqrt(2): x * (2^63/sqrt 2) / 2^64 * 2
            o << "    { const longlong2 t = kp.fxt[i]; T1[i] = make_longlong2(__mul64hi(t.x, kRsqrt2Q63) << 1, "
                 "__mul64hi(t.y, kRsqrt2Q63) << 1); }\n";
        else
            o << "    T1[i] = kp.fxt[i];\n";
        o << "    T2[i] = kp.fxt[256 + i];\n";
    } else {
        o << "    { const double2 e = kp.tw[i]; TW[i].x = (T)(e.x * " << dbl(table_scale) << "); TW[i].y = (T)(e.y * "
          << dbl(table_scale) << "); }\n";
    }
    for (int byte = 0; byte < 4; byte++) {
        o << "    OUTT[" << byte << "][i] = 0ull";
        for (int b = 0; b < 8; b++) {
            const int k = byte * 8 + b;
            if (k < P.n_outer)
                o << " | ((uint64_t)((i >> " << b << ") & 1) << " << (int)P.outer_bits[k] << ")";
        }
        o << ";\n";
    }
    o << "  }\n  __syncthreads();\n";
    emit_io_prologue(o, P, K, NT, E, n);
    // swizzle of an arbitrary tile index (perm rounds)
    o << "  auto swz = [](uint32_t v) -> uint32_t {\n    return 0u";
    for (int p = 0; p < K; p++) o << " ^ (((v >> " << p << ") & 1u) * " << hex32((uint32_t)swc(p)) << ")";
    o << ";\n  };\n  (void)swz;\n";
    o << "  long long tile = blockIdx.x;\n  int par = 0;\n  (void)Pf1;\n  if (tile < ntiles) prefetch(tile, Pf0);\n";
    if (two) o << "  if (tile + gridDim.x < ntiles) prefetch(tile + gridDim.x, Pf1);\n";
    if (hoist == 0) {
        o << "  if (tile < ntiles) {\n    const uint64_t xo = deposit(tile);\n";
        emit_slot_sums(o, S, P, S.rounds[P.round_begin], NT);
        o << "  }\n";
    }
    o << "  for (; tile < ntiles; tile += gridDim.x, par ^= " << (two ? 1 : 0) << ") {\n"
      << "    const uint64_t xo = deposit(tile);\n"
      << "    A *Pf = par ? Pf1 : Pf0;\n";
    if (fx) o << "    long long ar[16], ai[16];\n    uint32_t Sx = 0u;\n";
    else o << "    A a[16];\n";
    for (int r = 0; r < P.n_rounds; r++) {
        const DevRound &R = S.rounds[P.round_begin + r];
        o << "    { // round " << r << "\n";
        if (r == 0)
            o << (two ? "      if (tile + gridDim.x < ntiles) cp_async_wait_one(); else cp_async_wait_all();\n"
                      : "      cp_async_wait_all();\n");
        o << (warp_local_round(S, P, r, hoist) ? "      __syncwarp();\n" : "      __syncthreads();\n");
        if (!fx && r > 0 && r == pf_round) o << pf_next;
        if (R.n_diag > 0 && r != hoist) emit_round_staging(o, S, P, R, NT, dbl_state);
        o << "      const uint32_t lf = " << thread_expr(R, K, lcol, false) << ";\n"
          << "      const uint32_t sw = " << thread_expr(R, K, swc, false) << ";\n"
          << "      (void)lf; (void)sw;\n";
        if (r == 0 && fx) {
            // the tile's largest exponent, then the fixed-point conversion
            o << "      { double2 d[16];\n        uint32_t em = 0u;\n";
            for (int s = 0; s < 16; s++) {
                uint32_t l = 0;
                for (int i = 0; i < 4; i++)
                    if ((s >> i) & 1) l |= 1u << R.reg_pos[i];
                o << "        d[" << s << "] = Pf[lf | " << hex32(l) << "];\n"
                  << "        em = max(em, max(fx_exp(d[" << s << "].x), fx_exp(d[" << s << "].y)));\n";
            }
            o << "        em = __reduce_max_sync(0xffffffffu, em);\n"
              << "        if (lane == 0) EM[warp] = em;\n"
              << "        __syncthreads();\n"
              << "        Sx = EM[0];\n"
              << "        #pragma unroll\n"
              << "        for (int w = 1; w < NT / 32; w++) Sx = max(Sx, EM[w]);\n"
              << "        #pragma unroll\n"
              << "        for (int s = 0; s < 16; s++) { ar[s] = fx_from(d[s].x, Sx, " << fx_hr
              << "); ai[s] = fx_from(d[s].y, Sx, " << fx_hr << "); }\n"
              << "      }\n"
              << pf_next;
        } else if (r == 0) {
            for (int s = 0; s < 16; s++) {
                uint32_t l = 0;
                for (int i = 0; i < 4; i++)
                    if ((s >> i) & 1) l |= 1u << R.reg_pos[i];
                o << "      a[" << s << "] = Pf[lf | " << hex32(l) << "];\n";
            }
            if (pf_round == 0) o << "      __syncthreads();\n" << pf_next;
        } else {
            for (int s = 0; s < 16; s++) {
                uint32_t cs = 0;
                for (int i = 0; i < 4; i++)
                    if ((s >> i) & 1) cs ^= (uint32_t)swc(R.reg_pos[i]);
                if (fx)
                    o << "      { const longlong2 v = XI[sw ^ " << hex32(cs) << "]; ar[" << s << "] = v.x; ai[" << s
                      << "] = v.y; }\n";
                else
                    o << "      a[" << s << "] = X[sw ^ " << hex32(cs) << "];\n";
            }
        }
        if (hoist >= 0 && r == staging_round(P, hoist)) emit_hoisted_slot_sums(o, S, P, hoist, NT);
        int kph[16] = {0};   // fx: register s holds i^-kph[s] times its amplitude
        C64Rounds reps;      // complex64: the slots' representations
        reps.reset();
        // SD_C64_SCALAR=1 emits every butterfly as plain scalar code (the
        // reference the CPU tests compare the packed code with)
        const bool packed_bf = !fx && !getenv("SD_C64_SCALAR");
        // the last round's store folds the representations into its scale
        const bool store_folds = (R.flags & 2) && pass_scale != 1.0;
        bool need_xf = (R.flags & 2) != 0;
        for (int oi = R.op_begin; oi < R.op_end; oi++)
            need_xf |= S.ops[oi].kind == D_PHASE;
        if (need_xf) o << "      const uint64_t xf = xo | " << thread_expr(R, K, gbit, true) << ";\n";
        for (int oi = R.op_begin; oi < R.op_end; oi++) {
            const DevOp &op = S.ops[oi];
            if (op.kind == D_HAD && fx) {
                emit_had_fx(o, op.slot, c1_a(op.arg), c1_b(op.arg), kph);
            } else if (op.kind == D_MONO && fx) {
                emit_mono_fx(o, op.slot, c1_a(op.arg), c1_x(op.arg), kph);
            } else if (op.kind == D_HAD && packed_bf) {
                reps.had(o, S, R, oi, store_folds);
            } else if (op.kind == D_MONO && packed_bf) {
                reps.mono(o, op);
            } else if (op.kind == D_HAD) {
                o << "      had_fixed<" << op.slot << ", " << c1_a(op.arg) << ", " << c1_b(op.arg) << ">(a);\n";
            } else if (op.kind == D_MONO) {
                o << "      mono_fixed<" << op.slot << ", " << c1_a(op.arg) << ", " << c1_x(op.arg) << ">(a);\n";
            } else if (op.kind == D_PHASE) {
                if (packed_bf) reps.plain(o);
                o << "      { const int gq[4] = {" << (int)P.tile_bits[R.reg_pos[0]] << ", "
                  << (int)P.tile_bits[R.reg_pos[1]] << ", " << (int)P.tile_bits[R.reg_pos[2]] << ", "
                  << (int)P.tile_bits[R.reg_pos[3]] << "};\n"
                  << (fx ? "        fx_phase_apply(ar, ai, xf, gq, kp.phases[" : "        phase_apply(a, xf, gq, kp.phases[")
                  << op.arg << "], kp.mask_pool); }\n";
            } else {
                const DevDiag &d = S.diags[op.arg];
                const double sc = (op.pad && !table_scaled) ? P.scale : 1.0;
                o << "      { uint64_t G[16];\n";
                if (r == hoist) emit_class_sums_full(o, S, R, d, dbl_state ? 0ull : (1ull << 31));
                else emit_class_sums(o, S, R, d);
                if (fx)
                    o << "        wht16(G);\n"
                      << "        #pragma unroll\n"
                      << "        for (int s = 0; s < 16; s++) fx_rotate(ar[s], ai[s], G[s], T1, T2);\n"
                      << "      }\n";
                else if (packed_bf) {
                    reps.rotate(o, S, R, oi, sc);
                    o << "      }\n";
                } else
                    o << "        diag_rotate(a, G, TW, (T)" << dbl(sc) << ");\n"
                      << "      }\n";
            }
        }
        if (packed_bf && !store_folds) reps.plain(o);
        if (fx) {
            const int sh = fx_shift[r];
            if (sh > 0)
                o << "      #pragma unroll\n"
                  << "      for (int s = 0; s < 16; s++) { ar[s] = (ar[s] + " << (1ll << (sh - 1)) << "ll) >> " << sh
                  << "; ai[s] = (ai[s] + " << (1ll << (sh - 1)) << "ll) >> " << sh << "; }\n";
            for (int s2 = 0; s2 < 16; s2++)
                if (kph[s2]) o << "      fx_mul_ipow(ar[" << s2 << "], ai[" << s2 << "], " << kph[s2] << ");\n";
        }
        if ((R.flags & 2) && fx) {
            if (fx_res_store)
                o << "      #pragma unroll\n"
                  << "      for (int s = 0; s < 16; s++) { ar[s] = __mul64hi(ar[s], kRsqrt2Q63); ai[s] = __mul64hi(ai[s], kRsqrt2Q63); }\n";
            o << "      { const int U = (int)Sx - " << (1085 - fx_hr - (fx_res_store ? 1 : 0)) << ";\n";
            for (int s = 0; s < 16; s++) {
                uint64_t g = 0;
                for (int i = 0; i < 4; i++)
                    if ((s >> i) & 1) g |= gbit(R.reg_pos[i]);
                o << "        psi[xf | " << hex64(g) << "] = make_double2(fx_to(ar[" << s << "], U), fx_to(ai[" << s
                  << "], U));\n";
            }
            o << "      }\n";
        } else if (R.flags & 2) {
            for (int s = 0; s < 16; s++) {
                uint64_t g = 0;
                for (int i = 0; i < 4; i++)
                    if ((s >> i) & 1) g |= gbit(R.reg_pos[i]);
                if (pass_scale != 1.0 && packed_bf) {
                    // the slot's representation folded into the scale
                    const SlotRep &rp = reps.rep[s];
                    const std::string fr = dbl(rp.sr * pass_scale), fi = dbl(rp.si * pass_scale);
                    if (rp.sw == 0)
                        o << "      psi[xf | " << hex64(g) << "] = __fmul2_rn(a[" << s << "], make_float2((T)" << fr
                          << ", (T)" << fi << "));\n";
                    else
                        o << "      psi[xf | " << hex64(g) << "] = make_float2(a[" << s << "].y * (T)" << fr << ", a["
                          << s << "].x * (T)" << fi << ");\n";
                } else if (pass_scale != 1.0)
                    o << "      { A w = a[" << s << "]; w.x *= (T)" << dbl(pass_scale) << "; w.y *= (T)"
                      << dbl(pass_scale) << "; psi[xf | " << hex64(g) << "] = w; }\n";
                else
                    o << "      psi[xf | " << hex64(g) << "] = a[" << s << "];\n";
            }
        } else if (R.perm >= 0) {
            if (r > 0) o << "      __syncthreads();\n";
            o << "      { const DevPerm &pm = kp.perms[" << R.perm << "];\n"
              << "        uint32_t l = 0u;\n"
              << "        #pragma unroll\n"
              << "        for (int p = 0; p < K; p++) if ((lf >> p) & 1) l ^= pm.col[p];\n"
              << "        for (int k = 0; k < " << P.n_outer << "; k++) if ((tile >> k) & 1) l ^= pm.ocol[k];\n"
              << "        const uint32_t base = swz(l);\n"
              << "        const uint32_t c0 = swz(pm.col[" << (int)R.reg_pos[0] << "]), c1 = swz(pm.col["
              << (int)R.reg_pos[1] << "]), c2 = swz(pm.col[" << (int)R.reg_pos[2] << "]), c3 = swz(pm.col["
              << (int)R.reg_pos[3] << "]);\n"
              << "        #pragma unroll\n"
              << "        for (int s = 0; s < 16; s++) "
              << (fx ? "XI" : "X")
              << "[base ^ ((s & 1) ? c0 : 0u) ^ ((s & 2) ? c1 : 0u) ^ "
                 "((s & 4) ? c2 : 0u) ^ ((s & 8) ? c3 : 0u)] = "
              << (fx ? "make_longlong2(ar[s], ai[s])" : "a[s]") << ";\n"
              << "      }\n";
        } else {
            for (int s = 0; s < 16; s++) {
                uint32_t cs = 0;
                for (int i = 0; i < 4; i++)
                    if ((s >> i) & 1) cs ^= (uint32_t)swc(R.reg_pos[i]);
                if (fx)
                    o << "      XI[sw ^ " << hex32(cs) << "] = make_longlong2(ar[" << s << "], ai[" << s << "]);\n";
                else
                    o << "      X[sw ^ " << hex32(cs) << "] = a[" << s << "];\n";
            }
        }
        o << "    }\n";
    }
    o << "  }\n}\n\n";
    return o.str();
}

// Whether pass pi runs the paired complex64 code (gen_pass_packed): its
// schedule keeps tile position 0 in register slot 0, and no round of the
// pass applies a tile permutation or a quarter-turn layer.
bool packed_pass(const Schedule &S, int pi) {
    if (!S.pin0) return false;
    const DevPass &P = S.passes[pi];
    for (int r = 0; r < P.n_rounds; r++) {
        const DevRound &R = S.rounds[P.round_begin + r];
        if (R.reg_pos[0] != 0 || R.perm >= 0) return false;
        for (int oi = R.op_begin; oi < R.op_end; oi++)
            if (S.ops[oi].kind == D_PHASE) return false;
    }
    return true;
}

// (x, y) <- i^k (x, y) as text: the component expressions of i^k times the
// amplitude with components ax, ay.
void ipow_text(int k, const std::string &ax, const std::string &ay, std::string &x, std::string &y) {
    switch (k & 3) {
    case 0: x = ax; y = ay; break;
    case 1: x = "-(" + ay + ")"; y = ax; break;
    case 2: x = "-(" + ax + ")"; y = "-(" + ay + ")"; break;
    default: x = ay; y = "-(" + ax + ")"; break;
    }
}

// Generated complex64 pass in the paired layout.  A thread's 16 amplitudes
// form 8 pairs that differ only in tile position 0 (register slot 0); pair k
// holds register slots 1..3 = the bits of k as two float2 values, R[k] =
// (re, re) and I[k] = (im, im) of its two amplitudes.  A one-qubit Clifford
// on slots 1..3 then treats both amplitudes of a pair with one packed f32x2
// instruction per component; the exchange between rounds moves 16-byte
// pairs (8 per 128-byte row, paired swizzle); the rotation of a group
// exponential and the global loads and stores work on pairs.  Pair k is held
// as i^-kph[k] times its value (kph fixed at generation time, as in the
// fixed-point passes), so that the quarter-turn phases of S^b H S^a only
// choose adds or subtracts; they are applied before each write.
std::string gen_pass_packed(const Schedule &S, int pi, int n) {
    const DevPass &P = S.passes[pi];
    const int K = S.K;
    const int NT = 1 << (K - 4);
    const int E = 2;
    auto gbit = [&](int p) -> uint64_t { return (uint64_t)1 << P.tile_bits[p]; };
    auto lcol = [&](int p) -> uint64_t { return (uint64_t)1 << p; };
    auto ucol = [&](int p) -> uint64_t { return p == 0 ? 0 : (uint64_t)pair_swizzle_col(p); };
    const double pass_scale = P.scale_in_diag ? 1.0 : P.scale;
    int n_diag = 0;
    for (int r = 0; r < P.n_rounds; r++) {
        const DevRound &R = S.rounds[P.round_begin + r];
        for (int oi = R.op_begin; oi < R.op_end; oi++) n_diag += S.ops[oi].kind == D_DIAG;
    }
    const bool table_scaled = P.scale_in_diag && n_diag == 1;
    const double table_scale = table_scaled ? P.scale : 1.0;
    const int hoist = hoisted_stage_round(S, P);
    bool two = false;
    jit_pass_smem(S, P, 8, K, &two);
    const std::string pf_next = two ? "      if (tile + 2ll * gridDim.x < ntiles) prefetch(tile + 2ll * gridDim.x, Pf);\n"
                                    : "      if (tile + gridDim.x < ntiles) prefetch(tile + gridDim.x, Pf);\n";
    const int pf_round = prefetch_round(S, P, hoist);
    std::ostringstream o;
    o << "extern \"C\" __global__ void __launch_bounds__(" << NT << ") " << kernel_name(pi, false)
      << "(A *__restrict__ psi, sd::KParams kp) {\n"
      << "  using namespace sd;\n"
      << "  constexpr int K = " << K << ", NT = " << NT << ", E = " << E << ";\n"
      << "  extern __shared__ __align__(16) unsigned char smraw[];\n"
      << "  float4 *X4 = reinterpret_cast<float4 *>(smraw);\n"
      << "  A *Pf0 = reinterpret_cast<A *>(smraw) + (1 << K), *Pf1 = Pf0 + " << (two ? "(1 << K)" : "0") << ";\n"
      << "  StagedTerm *ST = reinterpret_cast<StagedTerm *>(Pf0 + " << (two ? 2 : 1) << " * (1 << K));\n"
      << "  uint64_t *TQ = reinterpret_cast<uint64_t *>(ST + " << (P.max_stage > 0 ? P.max_stage : 1) << ");\n"
      << "  (void)ST; (void)TQ;\n";
    if (P.term_cache)
        o << "  uint64_t *TCM = TQ + " << P.max_tot << ";\n"
          << "  int64_t *TCQ = reinterpret_cast<int64_t *>(TCM + " << P.term_count << ");\n"
          << "  cache_terms(kp, " << P.term_begin << ", " << P.term_count << ", TCM, TCQ, threadIdx.x, NT);\n";
    o << "  __shared__ float TC[512], TS[512];\n"
      << "  __shared__ uint64_t OUTT[4][256];\n"
      << "  __shared__ uint64_t CST[4];\n"
      << "  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;\n"
      << "  (void)lane; (void)warp;\n"
      << "  for (int i = tid; i < 512; i += NT) {\n"
      << "    const double2 e = kp.tw[256 + i];\n"
      << "    TC[i] = (float)(e.x * " << dbl(table_scale) << ");\n"
      << "    TS[i] = (float)(e.y * " << dbl(table_scale) << ");\n"
      << "    if (i < 256) {\n";
    for (int byte = 0; byte < 4; byte++) {
        o << "      OUTT[" << byte << "][i] = 0ull";
        for (int b = 0; b < 8; b++) {
            const int k = byte * 8 + b;
            if (k < P.n_outer) o << " | ((uint64_t)((i >> " << b << ") & 1) << " << (int)P.outer_bits[k] << ")";
        }
        o << ";\n";
    }
    o << "    }\n  }\n  __syncthreads();\n";
    emit_io_prologue(o, P, K, NT, E, n);
    o << "  const float2 M1 = make_float2(-1.f, -1.f);\n  (void)M1;\n"
      << "  long long tile = blockIdx.x;\n  int par = 0;\n  (void)Pf1;\n  if (tile < ntiles) prefetch(tile, Pf0);\n";
    if (two) o << "  if (tile + gridDim.x < ntiles) prefetch(tile + gridDim.x, Pf1);\n";
    if (hoist == 0) {
        o << "  if (tile < ntiles) {\n    const uint64_t xo = deposit(tile);\n";
        emit_slot_sums(o, S, P, S.rounds[P.round_begin], NT);
        o << "  }\n";
    }
    o << "  for (; tile < ntiles; tile += gridDim.x, par ^= " << (two ? 1 : 0) << ") {\n"
      << "    const uint64_t xo = deposit(tile);\n"
      << "    A *Pf = par ? Pf1 : Pf0;\n"
      << "    const float4 *Pf4 = reinterpret_cast<const float4 *>(Pf);\n"
      << "    float2 R[8], I[8];\n";
    // register slot i (1..3) <-> bit i-1 of the pair index k
    auto slot_sum = [&](const DevRound &R, int k, const std::function<uint64_t(int)> &col) {
        uint64_t v = 0;
        for (int i = 1; i < 4; i++)
            if ((k >> (i - 1)) & 1) v ^= col(R.reg_pos[i]);
        return v;
    };
    for (int r = 0; r < P.n_rounds; r++) {
        const DevRound &R = S.rounds[P.round_begin + r];
        o << "    { // round " << r << "\n";
        if (r == 0)
            o << (two ? "      if (tile + gridDim.x < ntiles) cp_async_wait_one(); else cp_async_wait_all();\n"
                      : "      cp_async_wait_all();\n");
        o << (warp_local_round(S, P, r, hoist) ? "      __syncwarp();\n" : "      __syncthreads();\n");
        if (r > 0 && r == pf_round) o << pf_next;
        if (R.n_diag > 0 && r != hoist) emit_round_staging(o, S, P, R, NT, false);
        o << "      const uint32_t lf = " << thread_expr(R, K, lcol, false) << ";\n"
          << "      const uint32_t swu = " << thread_expr(R, K, ucol, false) << ";\n"
          << "      (void)lf; (void)swu;\n";
        if (r == 0) {
            for (int k = 0; k < 8; k++)
                o << "      { const float4 v = Pf4[(lf | " << hex32((uint32_t)slot_sum(R, k, lcol))
                  << ") >> 1]; R[" << k << "] = make_float2(v.x, v.z); I[" << k << "] = make_float2(v.y, v.w); }\n";
            if (pf_round == 0) o << "      __syncthreads();\n" << pf_next;
        } else {
            for (int k = 0; k < 8; k++)
                o << "      { const float4 v = X4[swu ^ " << hex32((uint32_t)slot_sum(R, k, ucol)) << "]; R[" << k
                  << "] = make_float2(v.x, v.y); I[" << k << "] = make_float2(v.z, v.w); }\n";
        }
        if (R.flags & 2) o << "      const uint64_t xf = xo | " << thread_expr(R, K, gbit, true) << ";\n";
        if (hoist >= 0 && r == staging_round(P, hoist)) emit_hoisted_slot_sums(o, S, P, hoist, NT);
        int kph[8] = {0};
        for (int oi = R.op_begin; oi < R.op_end; oi++) {
            const DevOp &op = S.ops[oi];
            if ((op.kind == D_HAD || op.kind == D_MONO) && op.slot == 0) {
                // within each pair (one frame for both amplitudes): scalar code
                const int PA = c1_a(op.arg);
                for (int k = 0; k < 8; k++) {
                    const std::string ks = std::to_string(k);
                    std::string wx, wy;
                    ipow_text(PA, "R[" + ks + "].y", "I[" + ks + "].y", wx, wy);
                    if (op.kind == D_HAD) {
                        std::string tx, ty;
                        ipow_text(c1_b(op.arg), "dx", "dy", tx, ty);
                        o << "      { const float wx = " << wx << ", wy = " << wy << ";\n"
                          << "        const float sx = R[" << k << "].x + wx, sy = I[" << k << "].x + wy;\n"
                          << "        const float dx = fmaf(-2.f, wx, sx), dy = fmaf(-2.f, wy, sy);\n"
                          << "        R[" << k << "].x = sx; I[" << k << "].x = sy; R[" << k << "].y = " << tx
                          << "; I[" << k << "].y = " << ty << "; }\n";
                    } else if (c1_x(op.arg)) {
                        o << "      { const float wx = " << wx << ", wy = " << wy << ";\n"
                          << "        R[" << k << "].y = R[" << k << "].x; I[" << k << "].y = I[" << k << "].x; R["
                          << k << "].x = wx; I[" << k << "].x = wy; }\n";
                    } else {
                        o << "      { const float wx = " << wx << ", wy = " << wy << "; R[" << k << "].y = wx; I[" << k
                          << "].y = wy; }\n";
                    }
                }
            } else if (op.kind == D_HAD) {
                const int bit = 1 << (op.slot - 1);
                for (int k = 0; k < 8; k++) {
                    if (k & bit) continue;
                    const int t = k | bit;
                    const int m = (c1_a(op.arg) + kph[t] - kph[k]) & 3;
                    // w = i^m v in pair k's frame: component source and sign
                    const std::string vR = "R[" + std::to_string(t) + "]", vI = "I[" + std::to_string(t) + "]";
                    std::string srcR, srcI;
                    int sgR, sgI;
                    switch (m) {
                    case 0: srcR = vR; sgR = 1; srcI = vI; sgI = 1; break;
                    case 1: srcR = vI; sgR = -1; srcI = vR; sgI = 1; break;
                    case 2: srcR = vR; sgR = -1; srcI = vI; sgI = -1; break;
                    default: srcR = vI; sgR = 1; srcI = vR; sgI = -1; break;
                    }
                    auto add = [&](const std::string &u, const std::string &src, int sg) {
                        return sg > 0 ? "__fadd2_rn(" + u + ", " + src + ")" : "__ffma2_rn(" + src + ", M1, " + u + ")";
                    };
                    auto dd = [&](const std::string &src, int sg, const std::string &su) {
                        return "__ffma2_rn(" + src + ", make_float2(" + (sg > 0 ? "-2.f, -2.f" : "2.f, 2.f") + "), " + su +
                               ")";
                    };
                    const std::string uR = "R[" + std::to_string(k) + "]", uI = "I[" + std::to_string(k) + "]";
                    o << "      { const float2 sR = " << add(uR, srcR, sgR) << ", sI = " << add(uI, srcI, sgI) << ";\n"
                      << "        const float2 dR = " << dd(srcR, sgR, "sR") << ", dI = " << dd(srcI, sgI, "sI") << ";\n"
                      << "        " << uR << " = sR; " << uI << " = sI; " << vR << " = dR; " << vI << " = dI; }\n";
                    kph[t] = (c1_b(op.arg) + kph[k]) & 3;
                }
            } else if (op.kind == D_MONO) {
                const int bit = 1 << (op.slot - 1);
                for (int k = 0; k < 8; k++) {
                    if (k & bit) continue;
                    const int t = k | bit;
                    kph[t] = (kph[t] + c1_a(op.arg)) & 3;
                    if (c1_x(op.arg)) {
                        o << "      { const float2 tR = R[" << k << "], tI = I[" << k << "]; R[" << k << "] = R[" << t
                          << "]; I[" << k << "] = I[" << t << "]; R[" << t << "] = tR; I[" << t << "] = tI; }\n";
                        std::swap(kph[k], kph[t]);
                    }
                }
            } else {   // D_DIAG
                const DevDiag &d = S.diags[op.arg];
                const double sc = (op.pad && !table_scaled) ? P.scale : 1.0;
                o << "      { uint64_t G[16];\n";
                if (r == hoist) emit_class_sums_full(o, S, R, d, 1ull << 31);
                else emit_class_sums(o, S, R, d);
                o << "        uint32_t g[16];\n"
                  << "        #pragma unroll\n"
                  << "        for (int s = 0; s < 16; s++) g[s] = (uint32_t)(G[s] >> 32);\n"
                  << "        wht16(g);\n";
                for (int k = 0; k < 8; k++)
                    o << "        rotate_pair32(R[" << k << "], I[" << k << "], g[" << 2 * k << "], g[" << 2 * k + 1
                      << "], TC, TS, (float)" << dbl(sc) << ");\n";
                o << "      }\n";
            }
        }
        // back to the amplitudes' own frame (and the pass scale before a store)
        const double ws = (R.flags & 2) ? pass_scale : 1.0;
        for (int k = 0; k < 8; k++) {
            const std::string ks = std::to_string(k);
            const std::string f = ws == 1.0 ? "M1" : "make_float2((float)" + dbl(-ws) + ", (float)" + dbl(-ws) + ")";
            const std::string fp = "make_float2((float)" + dbl(ws) + ", (float)" + dbl(ws) + ")";
            switch (kph[k]) {
            case 0:
                if (ws != 1.0)
                    o << "      R[" << ks << "] = __fmul2_rn(R[" << ks << "], " << fp << "); I[" << ks
                      << "] = __fmul2_rn(I[" << ks << "], " << fp << ");\n";
                break;
            case 1:   // i (R + iI) = -I + iR
                o << "      { const float2 t = R[" << ks << "]; R[" << ks << "] = __fmul2_rn(I[" << ks << "], " << f
                  << "); I[" << ks << "] = " << (ws == 1.0 ? "t" : "__fmul2_rn(t, " + fp + ")") << "; }\n";
                break;
            case 2:
                o << "      R[" << ks << "] = __fmul2_rn(R[" << ks << "], " << f << "); I[" << ks << "] = __fmul2_rn(I["
                  << ks << "], " << f << ");\n";
                break;
            default:  // -i (R + iI) = I - iR
                o << "      { const float2 t = I[" << ks << "]; I[" << ks << "] = __fmul2_rn(R[" << ks << "], " << f
                  << "); R[" << ks << "] = " << (ws == 1.0 ? "t" : "__fmul2_rn(t, " + fp + ")") << "; }\n";
                break;
            }
        }
        if (R.flags & 2) {
            for (int k = 0; k < 8; k++)
                o << "      *reinterpret_cast<float4 *>(psi + (xf | " << hex64(slot_sum(R, k, gbit))
                  << ")) = make_float4(R[" << k << "].x, I[" << k << "].x, R[" << k << "].y, I[" << k << "].y);\n";
        } else {
            for (int k = 0; k < 8; k++)
                o << "      X4[swu ^ " << hex32((uint32_t)slot_sum(R, k, ucol)) << "] = make_float4(R[" << k << "].x, R["
                  << k << "].y, I[" << k << "].x, I[" << k << "].y);\n";
        }
        o << "    }\n";
    }
    o << "  }\n}\n\n";
    return o.str();
}

std::string cache_dir() {
    const char *e = getenv("SD_JIT_CACHE");
    if (e && *e) return e;
    const char *x = getenv("XDG_CACHE_HOME");
    if (x && *x) return std::string(x) + "/sd_jit";
    const char *h = getenv("HOME");
    return std::string(h && *h ? h : "/tmp") + "/.cache/sd_jit";
}

void mkdirs(const std::string &p) {
    std::string cur;
    std::stringstream ss(p);
    std::string part;
    if (!p.empty() && p[0] == '/') cur = "/";
    while (std::getline(ss, part, '/')) {
        if (part.empty()) continue;
        cur += part + "/";
        mkdir(cur.c_str(), 0755);
    }
}

std::string compile_cubin(const std::string &src, std::string &cubin) {
    nvrtcProgram prog;
    const char *hdrs[] = {kJitDevTypes, kJitFixedPoint, kJitTileDevice};
    const char *names[] = {"dev_types.h", "fixed_point.cuh", "tile_device.cuh"};
    if (g_nvrtc.create(&prog, src.c_str(), "sd_passes.cu", 3, hdrs, names) != NVRTC_SUCCESS)
        return "nvrtcCreateProgram failed";
    const char *opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "-lineinfo", "-DNDEBUG"};
    nvrtcResult rc = g_nvrtc.compile(prog, 4, opts);
    if (rc != NVRTC_SUCCESS) {
        size_t ls = 0;
        g_nvrtc.log_size(prog, &ls);
        std::string log(ls, '\0');
        if (ls) g_nvrtc.log(prog, &log[0]);
        g_nvrtc.destroy(&prog);
        return "NVRTC compile failed: " + log.substr(0, 2000);
    }
    size_t cs = 0;
    g_nvrtc.cubin_size(prog, &cs);
    cubin.assign(cs, '\0');
    g_nvrtc.cubin(prog, &cubin[0]);
    g_nvrtc.destroy(&prog);
    return "";
}

}  // namespace

bool jit_available(std::string *why) {
    std::lock_guard<std::mutex> lk(g_mu);
    init_locked();
    if (why) *why = g_why;
    return g_nvrtc.ok && g_drv.ok;
}

std::string source_range(const Schedule &S, int n, bool dbl_state, int first, int last) {
    std::ostringstream src;
    src << "#include \"dev_types.h\"\n#include \"tile_device.cuh\"\n"
        << "typedef " << (dbl_state ? "double" : "float") << " T;\n"
        << "typedef " << (dbl_state ? "double2" : "float2") << " A;\n\n";
    for (int p = first; p < last; p++)
        src << (!dbl_state && packed_pass(S, p) ? gen_pass_packed(S, p, n) : gen_pass(S, p, n, dbl_state));
    return src.str();
}

std::string jit_source(const Schedule &S, int n, bool dbl_state) {
    return source_range(S, n, dbl_state, 0, (int)S.passes.size());
}

std::string jit_compile_check(const std::string &src) {
    std::lock_guard<std::mutex> lk(g_mu);
    init_locked();
    if (!g_nvrtc.ok) return g_why;
    std::string cubin;
    return compile_cubin(src, cubin);
}

namespace {

constexpr int kChunk = 12;   // passes per NVRTC program

// Hash of the device headers the generated sources include: part of the
// cache key, so that cached kernels of an older library are not reused.
size_t headers_hash() {
    static const size_t h = std::hash<std::string>{}(std::string(kJitDevTypes) + kJitFixedPoint + kJitTileDevice);
    return h;
}

// Sources, cache keys and cubins of S's pass chunks: cubins come from the
// in-memory module table (left empty, mods[c] set), the disk cache, or NVRTC
// (compiled on a pool of host threads and written to the disk cache).
// Called with g_mu held.
std::string chunk_cubins(const Schedule &S, int n, bool dbl_state, std::vector<std::string> &key,
                         std::vector<std::string> &cubin, std::vector<CUmodule> *mods, int *compiled) {
    const int P = (int)S.passes.size();
    const int nchunks = (P + kChunk - 1) / kChunk;
    int maj = 0, min = 0;
    g_nvrtc.version(&maj, &min);
    std::vector<std::string> code(nchunks), err(nchunks);
    key.assign(nchunks, "");
    cubin.assign(nchunks, "");
    if (mods) mods->assign(nchunks, nullptr);
    const std::string dir = cache_dir();
    std::vector<int> todo;
    for (int c = 0; c < nchunks; c++) {
        code[c] = source_range(S, n, dbl_state, c * kChunk, std::min(P, (c + 1) * kChunk));
        key[c] = std::to_string(std::hash<std::string>{}(code[c])) + "_" + std::to_string(code[c].size()) +
                 "_h" + std::to_string(headers_hash()) + "_nvrtc" + std::to_string(maj) + "." + std::to_string(min);
        auto it = g_modules.find(key[c]);
        if (it != g_modules.end() && mods) {
            (*mods)[c] = it->second;
            continue;
        }
        std::ifstream f(dir + "/" + key[c] + ".cubin", std::ios::binary);
        if (f) cubin[c].assign(std::istreambuf_iterator<char>(f), std::istreambuf_iterator<char>());
        if (cubin[c].empty()) todo.push_back(c);
    }
    if (compiled) *compiled = (int)todo.size();
    if (!todo.empty()) {
        unsigned hw = std::thread::hardware_concurrency();
        const int nthreads = (int)std::max(1u, std::min<unsigned>(hw ? hw : 4, (unsigned)todo.size()));
        std::atomic<int> next{0};
        std::vector<std::thread> pool;
        for (int t = 0; t < nthreads; t++)
            pool.emplace_back([&]() {
                for (int i = next++; i < (int)todo.size(); i = next++) {
                    const int c = todo[i];
                    err[c] = compile_cubin(code[c], cubin[c]);
                }
            });
        for (auto &th : pool) th.join();
        mkdirs(dir);
        for (int c : todo) {
            if (!err[c].empty()) return err[c];
            const std::string path = dir + "/" + key[c] + ".cubin";
            const std::string tmp = path + ".tmp" + std::to_string(getpid());
            std::ofstream f(tmp, std::ios::binary);
            if (f) {
                f.write(cubin[c].data(), (std::streamsize)cubin[c].size());
                f.close();
                rename(tmp.c_str(), path.c_str());
            }
        }
    }
    return "";
}

}  // namespace

std::string jit_precompile(const Schedule &S, int n, bool dbl_state, int *compiled) {
    std::lock_guard<std::mutex> lk(g_mu);
    init_locked();
    if (!g_nvrtc.ok) return g_why.empty() ? "NVRTC unavailable" : g_why;
    std::vector<std::string> key, cubin;
    return chunk_cubins(S, n, dbl_state, key, cubin, nullptr, compiled);
}

// Passes are compiled in chunks (one NVRTC program each, on a pool of host
// threads); each chunk's cubin is cached in memory and on disk by the hash of
// its source.
std::string jit_build(const Schedule &S, int n, bool dbl_state, JitProgram &out) {
    std::lock_guard<std::mutex> lk(g_mu);
    init_locked();
    if (!(g_nvrtc.ok && g_drv.ok)) return g_why;
    const int P = (int)S.passes.size();
    const int chunk = kChunk;
    const int nchunks = (P + chunk - 1) / chunk;
    std::vector<std::string> key, cubin;
    std::vector<CUmodule> mods;
    std::string e = chunk_cubins(S, n, dbl_state, key, cubin, &mods, nullptr);
    if (!e.empty()) return e;
    for (int c = 0; c < nchunks; c++) {
        if (mods[c]) continue;
        if (g_drv.load(&mods[c], cubin[c].data()) != CUDA_SUCCESS) return "cuModuleLoadData failed";
        g_modules[key[c]] = mods[c];
    }
    out = JitProgram{};
    out.module = mods.empty() ? nullptr : (void *)mods[0];
    out.K = S.K;
    for (int p = 0; p < P; p++) {
        CUfunction f = nullptr;
        const std::string name = kernel_name(p, dbl_state);
        if (g_drv.get_function(&f, mods[p / chunk], name.c_str()) != CUDA_SUCCESS) return "missing kernel " + name;
        const size_t amp = dbl_state ? 16 : 8;
        const size_t smem = jit_pass_smem(S, S.passes[p], amp, S.K, nullptr);
        if (g_drv.set_attr(f, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, (int)smem) != CUDA_SUCCESS)
            return "cuFuncSetAttribute failed";
        int occ = 0;
        if (g_drv.occupancy(&occ, f, 1 << (S.K - 4), smem) != CUDA_SUCCESS) return "occupancy query failed";
        out.funcs.push_back((void *)f);
        out.occupancy.push_back(occ > 0 ? occ : 1);
        out.smem.push_back(smem);
    }
    return "";
}

cudaError_t jit_launch(const JitProgram &jp, int pass, void *psi, const KParams &kp, int n, int num_sms,
                       cudaStream_t st) {
    const int64_t ntiles = (int64_t)1 << (n - jp.K);
    int64_t grid = (int64_t)num_sms * jp.occupancy[pass];
    if (grid > ntiles) grid = ntiles;
    void *ps = psi;
    KParams k = kp;
    void *args[] = {&ps, &k};
    CUresult r = g_drv.launch((CUfunction)jp.funcs[pass], (unsigned)grid, 1, 1, 1u << (jp.K - 4), 1, 1,
                              (unsigned)jp.smem[pass], (CUstream)st, args, nullptr);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorLaunchFailure;
}

}  // namespace sd
