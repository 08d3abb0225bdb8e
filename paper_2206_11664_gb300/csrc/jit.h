// Run-time specialised tile passes (see jit.cpp).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "sd_internal.h"

namespace sd {

struct JitProgram {
    void *module = nullptr;          // CUmodule
    std::vector<void *> funcs;       // CUfunction per pass
    std::vector<int> occupancy;      // resident blocks per SM per pass
    std::vector<size_t> smem;        // dynamic shared memory per pass
    int K = 0;
    bool ok() const { return module != nullptr; }
};

// True if NVRTC and the driver entry points could be loaded; else why not.
bool jit_available(std::string *why);

// Generate, compile (or fetch from the cache) and load one kernel per pass of
// S.  Returns "" on success, else the reason (the caller then keeps using the
// interpreter kernel).
std::string jit_build(const Schedule &S, int n, bool dbl, JitProgram &out);

// Compile S's kernels into the disk cache without loading them (no GPU
// needed); *compiled (may be NULL) receives the number of chunks compiled.
std::string jit_precompile(const Schedule &S, int n, bool dbl, int *compiled);

// The generated source of S's kernels, and a compile-only check of it
// (returns "" or the compiler's log); both need no GPU.
std::string jit_source(const Schedule &S, int n, bool dbl);
std::string jit_compile_check(const std::string &src);

cudaError_t jit_launch(const JitProgram &jp, int pass, void *psi, const KParams &kp, int n,
                       int num_sms, cudaStream_t st);

}  // namespace sd
