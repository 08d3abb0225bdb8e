// Prints the CUDA source the run-time compiler would get for the complex64
// tile passes of one Trotter call, for the CPU tests of the pass generator.
//
// It plans with the library's host code (planner.cpp), builds `reps`
// unmerged steps (first order: groups in order; second order: the Strang
// sequence) as one circuit, canonicalises its one-qubit runs, schedules it
// (schedule.cpp) and prints jit_source() (jit.cpp) of the schedule.
//
// Usage: pass_source_dump <input>; the input is the schedule-only input of
// schedule_emulator.cpp: int32 n, int64 m, int32 skip_rule, int32 K, int32 c,
// int32 order, int32 reps, int64 steps (unused), float64 dt, uint64 x[m],
// uint64 z[m], float64 coeffs[m].
#include <cstdio>
#include <string>
#include <vector>

#include "jit.h"
#include "sd_internal.h"

namespace sd {
void set_last_error(const std::string &) {}
}  // namespace sd

using namespace sd;

int main(int argc, char **argv) {
    if (argc != 2) return 2;
    FILE *f = std::fopen(argv[1], "rb");
    if (!f) return 2;
    int32_t n, skip, K, c, order, reps;
    int64_t m, steps;
    double dt;
    bool ok = std::fread(&n, 4, 1, f) == 1 && std::fread(&m, 8, 1, f) == 1 && std::fread(&skip, 4, 1, f) == 1 &&
              std::fread(&K, 4, 1, f) == 1 && std::fread(&c, 4, 1, f) == 1 && std::fread(&order, 4, 1, f) == 1 &&
              std::fread(&reps, 4, 1, f) == 1 && std::fread(&steps, 8, 1, f) == 1 && std::fread(&dt, 8, 1, f) == 1;
    ok = ok && m > 0 && reps >= 1;
    std::vector<uint64_t> x(ok ? m : 0), z(ok ? m : 0);
    std::vector<double> coef(ok ? m : 0);
    ok = ok && std::fread(x.data(), 8, m, f) == (size_t)m && std::fread(z.data(), 8, m, f) == (size_t)m &&
         std::fread(coef.data(), 8, m, f) == (size_t)m;
    std::fclose(f);
    if (!ok) return 2;
    Plan plan;
    std::string e = make_plan(n, m, x.data(), z.data(), skip, plan);
    if (!e.empty()) {
        std::fprintf(stderr, "plan: %s\n", e.c_str());
        return 1;
    }
    const int G = (int)plan.groups.size();
    Circuit circ;
    for (int r = 0; r < reps; r++) {
        if (order == 1 || G == 1) {
            for (int g = 0; g < G; g++) append_group_step(plan, g, 1.0, dt, coef, circ);
        } else {
            for (int g = 0; g < G - 1; g++) append_group_step(plan, g, 0.5, dt, coef, circ);
            append_group_step(plan, G - 1, 1.0, dt, coef, circ);
            for (int g = G - 2; g >= 0; g--) append_group_step(plan, g, 0.5, dt, coef, circ);
        }
    }
    canonicalize_1q(circ, n);
    Schedule S;
    e = schedule_circuit(circ, n, K, c & 15, S, false, false);
    if (!e.empty()) {
        std::fprintf(stderr, "schedule: %s\n", e.c_str());
        return 1;
    }
    std::fputs(jit_source(S, n, false).c_str(), stdout);
    return 0;
}
