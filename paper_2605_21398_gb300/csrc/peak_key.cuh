// Per-rotation peak key shared by the plane passes: the ordered bits of the
// score in the high word and the complement of the canvas index in the low
// word, so that the largest key is the highest score and, among equal
// scores, the lowest linear canvas index (the tie rule of the argmax).
#pragma once
#include <stdint.h>

namespace dock {

__device__ __forceinline__ unsigned long long pack_key(float v, uint32_t idx)
{
    uint32_t u = __float_as_uint(__fadd_rn(v, 0.0f));   // -0 -> +0: equal scores compare equal
    uint32_t k = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return ((unsigned long long)k << 32) | (unsigned long long)(0xFFFFFFFFu - idx);
}

}  // namespace dock
