// Library-wide entry points of the C ABI: status names and version.
#include "common.cuh"

extern "C" const char* gpa_status_string(int status) {
    switch (status) {
        case GPA_OK: return "GPA_OK";
        case GPA_ERR_ARG: return "GPA_ERR_ARG: null pointer or size out of range";
        case GPA_ERR_INDEX: return "GPA_ERR_INDEX: an index outside its index set";
        case GPA_ERR_CUDA: return "GPA_ERR_CUDA: a CUDA launch or runtime call failed";
        case GPA_ERR_WORKSPACE: return "GPA_ERR_WORKSPACE: workspace smaller than required";
        case GPA_ERR_TIMEOUT: return "GPA_ERR_TIMEOUT: a bounded device wait gave up";
        case GPA_ERR_UNSUPPORTED: return "GPA_ERR_UNSUPPORTED: shape, precision or strategy not provided";
        case GPA_ERR_ALIGN: return "GPA_ERR_ALIGN: pointer lacks the required alignment";
    }
    return "unknown gpa_status";
}

extern "C" int gpa_version(void) { return 100; }
