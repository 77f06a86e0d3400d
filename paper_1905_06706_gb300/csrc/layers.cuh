// The weight layer of Sec. 3.1 without an FP64 division (the FP64 units are slow on
// GB300, and the reduction and the key kernels take it once per vertex).
#pragma once
#include "common.cuh"

namespace gg {

// floor(log2 of the correctly rounded quotient w / w_min), clamped to [0, 63]: the
// exponent of that quotient, which for normal w and w_min follows from the bit fields.
// With mantissas m_w, m_min in [1, 2), w / w_min = (m_w / m_min) 2^(e_w - e_min); the
// mantissa quotient lies in [1, 2 - 2^-52] when m_w >= m_min and in (1/2, 1 - 2^-53)
// otherwise, so it never rounds up to the next power of two, and scaling by 2^(e_w -
// e_min) is exact: the exponent is e_w - e_min - [m_w < m_min].  Outside the normal
// range (and for 0, inf, NaN) the quotient is formed.
GG_HD int layer_of_bits(double w, double w_min) {
    const uint64_t bw = double_to_bits(w), bm = double_to_bits(w_min);
    const int ew = (int)((bw >> 52) & 0x7ff), em = (int)((bm >> 52) & 0x7ff);
    if (ew == 0 || em == 0 || ew == 0x7ff || em == 0x7ff || (bw >> 63) || (bm >> 63))
        return layer_of(w, w_min);
    const uint64_t M = 0x000fffffffffffffULL;
    int layer = ew - em - ((bw & M) < (bm & M) ? 1 : 0);
    if (layer < 0) layer = 0;
    if (layer > kMaxLayers - 1) layer = kMaxLayers - 1;
    return layer;
}

}  // namespace gg
