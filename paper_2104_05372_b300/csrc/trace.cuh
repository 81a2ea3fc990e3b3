// Optional per-launch timing with CUDA events (off by default). When enabled
// with gpa_trace_enable(1), every kernel the library launches is bracketed by
// two events on its stream; gpa_trace_summary() resolves them per kernel name.
#pragma once

#include <cuda_runtime.h>

namespace gpa {
void trace_begin(const char* name, cudaStream_t s);
void trace_end(cudaStream_t s);
}  // namespace gpa

// Launch `launch` (a kernel launch statement) bracketed by trace events and
// check it; returns GPA_ERR_CUDA from the enclosing function on failure.
#define GPA_LAUNCH(name, stream, ...)        \
    do {                                     \
        gpa::trace_begin(name, stream);      \
        __VA_ARGS__;                         \
        gpa::trace_end(stream);              \
        GPA_LAUNCH_CHECK();                  \
    } while (0)
