// Length-256 (and, at the end, length-128) DFTs held in registers, 16 threads per sequence
// (256 = 16 x 16, Cooley-Tukey):
//   X[k1 + 16 k2] = sum_n2 w16^(n2 k2) w256^(n2 k1) sum_n1 x[16 n1 + n2] w16^(n1 k1),
// with w_N = e^{-2 pi i / N} (forward) or its conjugate (inverse). Thread n2 loads the 16
// elements x[16 n1 + n2] (consecutive threads read consecutive elements), runs a 16-point DFT in
// registers, applies the twiddles, exchanges through shared memory once (a 16 x 16 transpose)
// and runs the second 16-point DFT; it then holds X[n2 + 16 k2], k2 = 0..15, so stores are
// coalesced too. Each element passes through shared memory once per transform instead of once
// per radix stage.
#pragma once

#include "common.cuh"

namespace recon {

// u * w16^m, w16 = e^{-2 pi i / 16} (forward) or e^{+2 pi i / 16} (inverse), m compile-time.
template <int M, bool INV>
RECON_DEV float2 tw16(float2 u) {
    constexpr float c1 = 0.92387953251128675613f;  // cos(pi / 8)
    constexpr float s1 = 0.38268343236508977173f;  // sin(pi / 8)
    constexpr float h = 0.70710678118654752440f;
    constexpr int m = M & 15;
    float c, s;  // w = c - i s (forward); the inverse conjugates
    if constexpr (m == 0) return u;
    else if constexpr (m == 4) return mul_mi<INV>(u);
    else if constexpr (m == 8) return make_float2(-u.x, -u.y);
    else if constexpr (m == 12) return mul_mi<!INV>(u);
    else {
        switch (m) {
            case 1: c = c1; s = s1; break;
            case 2: c = h; s = h; break;
            case 3: c = s1; s = c1; break;
            case 5: c = -s1; s = c1; break;
            case 6: c = -h; s = h; break;
            case 7: c = -c1; s = s1; break;
            case 9: c = -c1; s = -s1; break;
            case 10: c = -h; s = -h; break;
            case 11: c = -s1; s = -c1; break;
            case 13: c = s1; s = -c1; break;
            case 14: c = h; s = -h; break;
            default: c = c1; s = -s1; break;  // 15
        }
        if (INV) s = -s;
        // (u.x + i u.y)(c - i s)
        return make_float2(fmaf(u.x, c, u.y * s), fmaf(u.y, c, -u.x * s));
    }
}

template <int N2, bool INV>
RECON_DEV void dft16_twiddle_row(float2 (&y)[16], const float2 (&a)[4]) {
    y[4 * N2 + 0] = a[0];
    y[4 * N2 + 1] = tw16<N2 * 1, INV>(a[1]);
    y[4 * N2 + 2] = tw16<N2 * 2, INV>(a[2]);
    y[4 * N2 + 3] = tw16<N2 * 3, INV>(a[3]);
}

// In-place 16-point DFT in natural order: u[k] = sum_n u[n] w16^(n k) (4 x 4 split).
template <bool INV>
RECON_DEV void dft16(float2 (&u)[16]) {
    float2 y[16];
    {
        float2 a[4] = {u[0], u[4], u[8], u[12]};
        SmallDFT<4, INV>::run(a);
        dft16_twiddle_row<0, INV>(y, a);
    }
    {
        float2 a[4] = {u[1], u[5], u[9], u[13]};
        SmallDFT<4, INV>::run(a);
        dft16_twiddle_row<1, INV>(y, a);
    }
    {
        float2 a[4] = {u[2], u[6], u[10], u[14]};
        SmallDFT<4, INV>::run(a);
        dft16_twiddle_row<2, INV>(y, a);
    }
    {
        float2 a[4] = {u[3], u[7], u[11], u[15]};
        SmallDFT<4, INV>::run(a);
        dft16_twiddle_row<3, INV>(y, a);
    }
    // y[4 n2 + k1] = w16^(n2 k1) sum_n1 u[4 n1 + n2] w4^(n1 k1); now the DFT over n2
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        float2 b[4] = {y[k1], y[4 + k1], y[8 + k1], y[12 + k1]};
        SmallDFT<4, INV>::run(b);
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) u[k1 + 4 * k2] = b[k2];
    }
}

// Shared-memory table tw2[k1 * 16 + j] = w256^(j k1) (forward sign), built from the length-256
// table tw[i] = e^{-2 pi i i / 256}; 256 entries, filled by the calling block.
RECON_DEV void fill_tw256(float2* tw2, const float2* __restrict__ tw_g) {
    for (int e = threadIdx.x; e < 256; e += blockDim.x) tw2[e] = tw_g[(e / 16) * (e % 16)];
}

// Twiddle step between the two 16-point stages: u[k1] *= w256^(j k1).
template <bool INV>
RECON_DEV void twiddle256(float2 (&u)[16], const float2* tw2, int j) {
#pragma unroll
    for (int k1 = 1; k1 < 16; ++k1) {
        float2 w = tw2[k1 * 16 + j];
        if (INV) w.y = -w.y;
        u[k1] = cmul(u[k1], w);
    }
}

// Length-256 DFT of one row held by the 16 lanes of a half-warp, lane j holding x[16 n1 + j]
// in u[n1]; on return u[k2] = X[j + 16 k2]. `sx` is the row's private 16 x 17 exchange buffer.
template <bool INV>
RECON_DEV void row_dft256(float2 (&u)[16], float2* sx, const float2* tw2, int j) {
    dft16<INV>(u);
    twiddle256<INV>(u, tw2, j);
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) sx[k1 * 17 + j] = u[k1];
    __syncwarp();
#pragma unroll
    for (int n2 = 0; n2 < 16; ++n2) u[n2] = sx[j * 17 + n2];
    __syncwarp();
    dft16<INV>(u);
}

// ---- length 128 = 16 x 8, 8 threads per sequence ----
//   X[k1 + 16 k2] = sum_j w8^(j k2) w128^(j k1) sum_n1 x[8 n1 + j] w16^(n1 k1).
// Lane j loads x[8 n1 + j] (n1 < 16), runs the 16-point DFT and the twiddles, writes its 16
// values to the row's exchange buffer (16 x 9, row k1), and reads back rows 2j and 2j + 1 for
// two 8-point DFTs: it then holds X[2j + 16 k2] in a[k2] and X[2j + 1 + 16 k2] in b[k2].
constexpr int kX128 = 152;  // float2 per exchange buffer (16 x 9 + 8: alternate 16-bank offset)

// tw8[k1 * 8 + j] = w128^(j k1) (forward sign) from the length-128 table; 128 entries.
RECON_DEV void fill_tw128(float2* tw8, const float2* __restrict__ tw_g) {
    for (int e = threadIdx.x; e < 128; e += blockDim.x) tw8[e] = tw_g[(e / 8) * (e % 8)];
}

template <bool INV>
RECON_DEV void row_dft128(float2 (&u)[16], float2 (&a)[8], float2 (&b)[8], float2* sx,
                          const float2* tw8, int j) {
    dft16<INV>(u);
#pragma unroll
    for (int k1 = 1; k1 < 16; ++k1) {
        float2 w = tw8[k1 * 8 + j];
        if (INV) w.y = -w.y;
        u[k1] = cmul(u[k1], w);
    }
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) sx[k1 * 9 + j] = u[k1];
    __syncwarp();
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
        a[jj] = sx[(2 * j) * 9 + jj];
        b[jj] = sx[(2 * j + 1) * 9 + jj];
    }
    __syncwarp();
    SmallDFT<8, INV>::run(a);
    SmallDFT<8, INV>::run(b);
}

}  // namespace recon
