// Opt-in launch timing for the roofline report: when a kernel class is
// enabled, its launches are bracketed by CUDA events on the launching stream
// and tagged with the launch's algorithmic FLOPs and bytes.
#pragma once
#include "common.cuh"

namespace ttsg {

enum ProfClass { PROF_GEMM = 0, PROF_QR = 1, PROF_SVD = 2, PROF_LSTSQ = 3, PROF_MISC = 4,
                 PROF_GRAM = 5, PROF_CHOL = 6, PROF_TC = 7, PROF_NCLASS = 8 };

bool prof_on(int cls);
// Counts every kernel launch the library enqueues (read by tt_launch_count).
void count_launch();
// Returns a token for prof_end (or -1 when the class is disabled).
int prof_begin(int cls, cudaStream_t st);
void prof_end(int token, cudaStream_t st, double flops, double bytes);

}  // namespace ttsg
