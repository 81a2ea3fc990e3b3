// Layout of an index plan (stable sort of element ids by a data-derived key).
#pragma once

#include <stddef.h>
#include <stdint.h>

namespace gpa {

struct PlanView {
    int64_t* header;      // {n_elems, n_keys, n_valid, reserved}
    int32_t* perm;        // element ids in key order
    int32_t* key_sorted;  // keys in that order (n_keys marks an invalid element)
    int32_t* aux_sorted;  // second index in that order
    int32_t* seg_off;     // [n_keys + 1]
};

inline size_t plan_a256(size_t v) { return (v + 255) & ~(size_t)255; }

inline size_t plan_size(int64_t n, int32_t n_keys) {
    size_t off = 256;  // header
    off += 3 * plan_a256(sizeof(int32_t) * (size_t)n);
    off += plan_a256(sizeof(int32_t) * ((size_t)n_keys + 1));
    return off;
}

inline PlanView plan_view(const void* plan, int64_t n, int32_t n_keys) {
    (void)n_keys;
    char* b = (char*)plan;
    PlanView v;
    v.header = (int64_t*)b;
    size_t off = 256;
    v.perm = (int32_t*)(b + off);       off += plan_a256(sizeof(int32_t) * (size_t)n);
    v.key_sorted = (int32_t*)(b + off); off += plan_a256(sizeof(int32_t) * (size_t)n);
    v.aux_sorted = (int32_t*)(b + off); off += plan_a256(sizeof(int32_t) * (size_t)n);
    v.seg_off = (int32_t*)(b + off);
    return v;
}

}  // namespace gpa
