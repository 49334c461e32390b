// qs_real2.cu -- finite-width beam on a periodic transverse grid (sm_103a).
//
// Narrow beams (Sec. IV.B: self-modulation and hosing) need the transverse
// profile n_b0(y, z) in real space.  Per slow-time step:
//   A. plasma response per transverse point, (d_xi^2 + 1) n_p = q n_b
//      (Eq. 5, local in r_perp): one thread per point marches xi with the
//      exact cell propagator and writes n_p at the cell centres;
//   B. per xi slice, the screened Poisson solve of Eq. (14),
//      Psi^ = n_p^ / (1 + k^2), and grad_perp Psi by spectral derivatives,
//      with hand-written FFTs: at N = 256 register four-step transforms by
//      16-thread teams (k_rowfft256, k_colfft256, k_rowinv_push256), at
//      N = 32..128 radix-2 Stockham transforms in shared memory:
//        K1  row FFTs along z (two real rows packed per complex FFT) ->
//            half spectrum S1 [xi][y][N/2+1] ([xi][N/2+1][y] at N = 256);
//        K2  column FFTs along y, multiply by kappa and i k_y kappa, two
//            inverse column FFTs -> T1 = Psi~, T2 = (d_y Psi)~ (same layout);
//        K3  inverse row FFTs (Psi and d_z Psi packed as real/imag of one
//            FFT, d_y Psi of two rows packed in another) fused with the push
//            d_tau G = -(q/(m gamma)) [n_b0 (Psi - n_p) + grad n_b0 . grad Psi],
//            n_b += dt G (kick-drift leapfrog, first kick dt/2).
// The gamma^-3 term is dropped here (gamma_b >> 1 for narrow-beam cases).
// State and intermediates are FP32; the state is laid out [xi][y][z] with z
// fastest.  At N = 256 the half spectra are column-major, so the column
// transforms move whole columns as contiguous runs and the row kernels do
// the transposition in the shared-memory staging they need anyway.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <string>
#include <vector>

#include "qs.h"
#include "qs_nvtx.h"

namespace r2 {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// twiddles tw[t] = exp(-2 pi i t / N), t < N/2
template <int N>
__device__ __forceinline__ void make_twiddles(float2 *tw) {
    for (int t = threadIdx.x; t < N / 2; t += blockDim.x) {
        float s, c;
        sincospif(-2.0f * t / N, &s, &c);
        tw[t] = make_float2(c, s);
    }
}

// Stockham radix-2 FFT of `rows` rows of length N stored at src[r * N + x];
// dst is scratch of the same size.  Returns the buffer holding the result.
// inverse: conjugate twiddles (no normalisation).
template <int N>
__device__ float2 *fft_rows(float2 *src, float2 *dst, int rows, const float2 *tw, bool inverse) {
    constexpr int H = N / 2;
    for (int m = 1; m < N; m <<= 1) {
        const int tstride = N / (2 * m);
        for (int idx = threadIdx.x; idx < rows * H; idx += blockDim.x) {
            const int r = idx / H, jj = idx - r * H;
            const int k = jj % m, g = jj / m;
            const float2 x0 = src[r * N + g * m + k];
            const float2 x1 = src[r * N + g * m + k + H];
            float2 w = tw[k * tstride];
            if (inverse) w.y = -w.y;
            const float2 y = cmul(w, x1);
            dst[r * N + g * 2 * m + k] = make_float2(x0.x + y.x, x0.y + y.y);
            dst[r * N + g * 2 * m + k + m] = make_float2(x0.x - y.x, x0.y - y.y);
        }
        __syncthreads();
        float2 *t = src; src = dst; dst = t;
    }
    return src;
}

// ---------------------------------------------------------------------------
// 256-point FFT by a team of 16 threads (four-step, 256 = 16 x 16): thread t
// holds x[t + 16 m] (m = 0..15), does a 16-point DFT over m in registers,
// multiplies by W256^(t k1), exchanges through a padded [16][17] buffer, and
// does the 16-point DFT over t; thread t then holds X[t + 16 k2].  The
// 16-point DFT is radix 4 x 4.  The inter-step twiddles W256^(t k1),
// W256 = exp(-2 pi i / 256), sit at tw[k1 * 17 + t] (TWN entries), so the
// 16 threads of a team read 16 consecutive entries.
// ---------------------------------------------------------------------------
// complex add and subtract as packed FP32x2 operations (a - b = fma(b, -1, a),
// rounded exactly like the subtraction)
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }

template <bool INV>
__device__ __forceinline__ void dft4(float2 &a0, float2 &a1, float2 &a2, float2 &a3) {
    const float2 t0 = add2(a0, a2), t1 = sub2(a0, a2), t2 = add2(a1, a3), t3 = sub2(a1, a3);
    a0 = add2(t0, t2);
    a2 = sub2(t0, t2);
    // t1 -/+ i t3 (forward: -i t3 = (t3.y, -t3.x))
    if (INV) {
        a1 = make_float2(t1.x - t3.y, t1.y + t3.x);
        a3 = make_float2(t1.x + t3.y, t1.y - t3.x);
    } else {
        a1 = make_float2(t1.x + t3.y, t1.y - t3.x);
        a3 = make_float2(t1.x - t3.y, t1.y + t3.x);
    }
}

constexpr int TWN = 16 * 17;

// a W16^k, W16 = exp(-2 pi i / 16) (conjugate when INV), for the k = b r
// (b, r < 4) of a radix-4 x 4 16-point DFT; k is a constant once the
// callers' loops are unrolled, so the multiplier folds to literals
template <bool INV>
__device__ __forceinline__ float2 w16mul(float2 a, int k) {
    constexpr float C1 = 0.923879532511286756f, S1 = 0.382683432365089772f, R2 = 0.707106781186547524f;
    float c, s;   // W16^k = (c, -s)
    switch (k) {
    case 0: return a;
    case 4: return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
    case 1: c = C1; s = S1; break;
    case 2: c = R2; s = R2; break;
    case 3: c = S1; s = C1; break;
    case 6: c = -R2; s = R2; break;
    default: c = -C1; s = -S1; break;   // k = 9
    }
    return cmul(a, make_float2(c, INV ? s : -s));
}

// x[k] <- sum_m x[m] W16^(m k) (conjugate twiddles when INV)
template <bool INV>
__device__ __forceinline__ void dft16(float2 (&x)[16]) {
    float2 y[16];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        float2 a0 = x[b], a1 = x[4 + b], a2 = x[8 + b], a3 = x[12 + b];
        dft4<INV>(a0, a1, a2, a3);
        y[4 * b + 0] = a0;
        y[4 * b + 1] = w16mul<INV>(a1, b);
        y[4 * b + 2] = w16mul<INV>(a2, 2 * b);
        y[4 * b + 3] = w16mul<INV>(a3, 3 * b);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        float2 a0 = y[c], a1 = y[4 + c], a2 = y[8 + c], a3 = y[12 + c];
        dft4<INV>(a0, a1, a2, a3);
        x[c] = a0; x[c + 4] = a1; x[c + 8] = a2; x[c + 12] = a3;
    }
}

// 256-point FFT of values held by a 16-thread team: on entry x[m] is entry
// t + 16 m, on return x[k] is entry t + 16 k of the transform.  T is the
// team's [16][17] exchange buffer; every thread of the warp must call it
// (both half-warp teams in step), and T may hold the inputs the team has
// just read (the entry barrier orders those reads before the writes).
// TWP: only W^t, W^2t, W^4t and W^8t are read from the table and the other
// inter-step twiddles are formed as products of them (at most two
// multiplications deep, a few ulp), for kernels whose shared-memory pipe is
// their limit.
template <bool INV, bool TWP = false>
__device__ __forceinline__ void fft256_reg(float2 (&x)[16], float2 *T, const float2 *tw256, int t) {
    dft16<INV>(x);
    __syncwarp();
    T[t] = x[0];   // W256^0
    if constexpr (TWP) {
        auto ld = [&](int k1) {
            float2 w = tw256[k1 * 17 + t];
            if (INV) w.y = -w.y;
            return w;
        };
        const float2 w1 = ld(1), w2 = ld(2), w4 = ld(4), w8 = ld(8);
        // w_k for k < 8, and w_(k + 8) = w_k w8
        auto put = [&](int k1, float2 w) {
            T[k1 * 17 + t] = cmul(x[k1], w);
            T[(k1 + 8) * 17 + t] = cmul(x[k1 + 8], cmul(w, w8));
        };
        T[8 * 17 + t] = cmul(x[8], w8);
        put(1, w1);
        put(2, w2);
        put(3, cmul(w1, w2));
        put(4, w4);
        put(5, cmul(w1, w4));
        const float2 w6 = cmul(w2, w4);
        put(6, w6);
        put(7, cmul(w1, w6));
    } else {
#pragma unroll
        for (int k1 = 1; k1 < 16; ++k1) {
            float2 w = tw256[k1 * 17 + t];
            if (INV) w.y = -w.y;
            T[k1 * 17 + t] = cmul(x[k1], w);
        }
    }
    __syncwarp();
#pragma unroll
    for (int tt = 0; tt < 16; ++tt) x[tt] = T[t * 17 + tt];
    dft16<INV>(x);
    __syncwarp();
}

// in-place FFT of one 256-entry row in shared memory by a 16-thread team
template <bool INV>
__device__ __forceinline__ void fft256_team(float2 *row, float2 *T, const float2 *tw256, int t) {
    float2 x[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) x[m] = row[t + 16 * m];
    fft256_reg<INV>(x, T, tw256, t);
#pragma unroll
    for (int k2 = 0; k2 < 16; ++k2) row[t + 16 * k2] = x[k2];
    __syncwarp();
}

__device__ __forceinline__ void make_tw256(float2 *tw) {
    for (int j = threadIdx.x; j < 256; j += blockDim.x) {
        const int k1 = j >> 4, t = j & 15;
        float s, c;
        sincospif(-2.0f * (float)(t * k1) / 256.0f, &s, &c);
        tw[k1 * 17 + t] = make_float2(c, s);
    }
}

// only the rows k1 = 1, 2, 4, 8 that the product-twiddle transforms read
__device__ __forceinline__ void make_tw256_p2(float2 *tw) {
    for (int j = threadIdx.x; j < 64; j += blockDim.x) {
        const int k1 = 1 << (j >> 4), t = j & 15;
        float s, c;
        sincospif(-2.0f * (float)(t * k1) / 256.0f, &s, &c);
        tw[k1 * 17 + t] = make_float2(c, s);
    }
}

// K1 for N = 256: 32 rows (16 packed) per CTA, 16 teams.  S1 is stored
// column-major, [xi][k_z][y], so that the column transforms read and write
// whole 256-entry columns as contiguous runs.
__global__ void __launch_bounds__(256, 5) k_rowfft256(const float *__restrict__ np, float2 *__restrict__ S1) {
    constexpr int N = 256, NH = 129, PR = 16, LA = 274;   // LA: packed-row stride (16-byte aligned, room for the exchange)
    extern __shared__ float2 sm[];
    float2 *tw = sm, *A = sm + TWN;
    const long long slice = blockIdx.y;
    const int r0 = blockIdx.x * 2 * PR;
    const int team = threadIdx.x >> 4, t = threadIdx.x & 15;
    make_tw256(tw);
    const float *src = np + slice * (long long)N * N;
    // 16-byte asynchronous copies, all in flight at once: rows r0 + 2 pr and
    // r0 + 2 pr + 1 land side by side (as floats) in packed row pr
    for (int i = threadIdx.x; i < 2 * PR * N / 4; i += blockDim.x) {
        const int row = i >> 6, c4 = i & 63;
        float *d = reinterpret_cast<float *>(A + (row >> 1) * LA) + (row & 1) * N + 4 * c4;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(d)),
                     "l"(src + (long long)(r0 + row) * N + 4 * c4) : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    {
        // team pr: the complex row (row 2 pr) + i (row 2 pr + 1), transformed in place
        const float *rf = reinterpret_cast<const float *>(A + team * LA);
        float2 x[16];
#pragma unroll
        for (int m = 0; m < 16; ++m) x[m] = make_float2(rf[t + 16 * m], rf[N + t + 16 * m]);
        fft256_reg<false>(x, A + team * LA, tw, t);   // exchange in the team's own row (read above)
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) A[team * LA + t + 16 * k2] = x[k2];
    }
    __syncthreads();
    // split each packed transform into its two rows' half spectra; the two
    // rows' entries at one k_z are neighbours in S1 (one 16-byte store), and
    // a warp stores 256 contiguous bytes for each of two k_z
    float2 *dst = S1 + slice * (long long)N * NH + r0;
    for (int i = threadIdx.x; i < PR * NH; i += blockDim.x) {
        const int pr = i & (PR - 1), k = i >> 4;
        const float2 Z = A[pr * LA + k], Zc = A[pr * LA + ((N - k) & (N - 1))];
        __stcg(reinterpret_cast<float4 *>(dst + (long long)k * N + 2 * pr),
               make_float4(0.5f * (Z.x + Zc.x), 0.5f * (Z.y - Zc.y), 0.5f * (Z.y + Zc.y), -0.5f * (Z.x - Zc.x)));
    }
}

// K2 for N = 256: 128 threads = 8 teams, spectral columns 8 b .. 8 b + 7 of
// one slice, one per team.  Columns 0 and 128 (k_z = 0 and the Nyquist
// column) are real sequences along y, so team 0 of block 0 transforms them
// as the real and imaginary parts of one complex column and 16 blocks cover
// the 129 columns.  S1, T1 and T2 are column-major ([xi][k_z][y]): a team
// loads its column straight into registers (16 threads read 128 contiguous
// bytes per access, a warp's two teams 256), keeps it there through the
// forward transform, the kappa and i k_y kappa products and both inverse
// transforms, and stores the results the same way; shared memory holds only
// the twiddles and the transforms' exchange buffers.
__global__ void __launch_bounds__(128, 5) k_colfft256(const float2 *__restrict__ S1, float2 *__restrict__ T1,
                                                      float2 *__restrict__ T2, float ly, float lz) {
    constexpr int N = 256, NH = 129, CB = 8, TSZ = 272;
    extern __shared__ float2 sm[];
    float2 *tw = sm, *Ts = sm + TWN + (threadIdx.x >> 4) * TSZ;
    const long long so = blockIdx.y * (long long)N * NH;
    const int c0 = blockIdx.x * CB;
    const int tm = threadIdx.x >> 4, t = threadIdx.x & 15, warp = threadIdx.x >> 5;
    const bool first = blockIdx.x == 0;
    const bool pk = first && tm == 0;            // columns 0 and 128 packed
    const bool w0 = first && warp == 0;          // (warp-uniform) the warp holding the packed pair
    const float2 *src = S1 + so + (long long)(c0 + tm) * N + t;
    float2 x[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) x[m] = __ldcs(src + 16 * m);
    if (pk) {
        const float *nq = reinterpret_cast<const float *>(S1 + so + 128LL * N + t);   // the Nyquist column (real)
#pragma unroll
        for (int m = 0; m < 16; ++m) x[m].y = __ldcs(nq + 32 * m);
    }
    make_tw256_p2(tw);
    __syncthreads();
    fft256_reg<false, true>(x, Ts, tw, t);
    // the packed pair needs X at -j: entry (256 - t - 16 k) % 256 sits in
    // thread (16 - t) % 16 at index 15 - k (t > 0) or (16 - k) % 16 (t = 0)
    if (w0) {
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) Ts[t * 17 + k2] = x[k2];
        __syncwarp();
    }
    const int pt = (16 - t) & 15;
    const float inv = 1.0f / (256.0f * 256.0f);
    const float ty = 6.283185307179586f / ly, tz = 6.283185307179586f / lz;
    const float kzv = tz * (float)(c0 + tm);
    float2 D[16];
    // (kappa to within 2 ulp: __fdividef; the branch is uniform in all but one warp)
    if (pk) {
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) {
            const int j = t + 16 * k2;
            const float ky = ty * (float)(j < 128 ? j : j - 256), kyd = j == 128 ? 0.0f : ky;
            // F0 = (X + conj Xm) / 2 (column 0), F1 = (X - conj Xm) / 2i (column 128)
            const float2 X = x[k2], Xm = Ts[pt * 17 + (t == 0 ? ((16 - k2) & 15) : 15 - k2)];
            const float2 F0 = make_float2(0.5f * (X.x + Xm.x), 0.5f * (X.y - Xm.y));
            const float2 F1 = make_float2(0.5f * (X.y + Xm.y), -0.5f * (X.x - Xm.x));
            const float kzn = tz * -128.0f;
            const float k0 = __fdividef(inv, 1.0f + ky * ky), k1 = __fdividef(inv, 1.0f + ky * ky + kzn * kzn);
            const float2 P0 = make_float2(k0 * F0.x, k0 * F0.y), P1 = make_float2(k1 * F1.x, k1 * F1.y);
            const float2 D0 = make_float2(-kyd * P0.y, kyd * P0.x), D1 = make_float2(-kyd * P1.y, kyd * P1.x);
            x[k2] = make_float2(P0.x - P1.y, P0.y + P1.x);   // P0 + i P1
            D[k2] = make_float2(D0.x - D1.y, D0.y + D1.x);   // D0 + i D1
        }
    } else {
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) {
            const int j = t + 16 * k2;
            const float ky = ty * (float)(j < 128 ? j : j - 256), kyd = j == 128 ? 0.0f : ky;
            const float kap = __fdividef(inv, 1.0f + ky * ky + kzv * kzv);
            const float2 P = make_float2(kap * x[k2].x, kap * x[k2].y);
            x[k2] = P;
            D[k2] = make_float2(-kyd * P.y, kyd * P.x);
        }
    }
    if (w0) __syncwarp();   // the exchange buffer is read before the transforms reuse it
    fft256_reg<true, true>(x, Ts, tw, t);
    fft256_reg<true, true>(D, Ts, tw, t);
    // entry y = t + 16 k2 of the column: columns 0 and 128 of the packed pair
    // are the real and imaginary parts
    float2 *d1 = T1 + so + (long long)(c0 + tm) * N + t, *d2 = T2 + so + (long long)(c0 + tm) * N + t;
    if (pk) {
        float2 *e1 = T1 + so + 128LL * N + t, *e2 = T2 + so + 128LL * N + t;
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) {
            __stcg(d1 + 16 * k2, make_float2(x[k2].x, 0.0f));
            __stcg(e1 + 16 * k2, make_float2(x[k2].y, 0.0f));
            __stcg(d2 + 16 * k2, make_float2(D[k2].x, 0.0f));
            __stcg(e2 + 16 * k2, make_float2(D[k2].y, 0.0f));
        }
    } else {
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) {
            __stcg(d1 + 16 * k2, x[k2]);
            __stcg(d2 + 16 * k2, D[k2]);
        }
    }
}

// signed spectral index and its derivative version (Nyquist zeroed)
template <int N>
__device__ __forceinline__ float sidx(int j) { return (float)(j < N / 2 ? j : j - N); }
template <int N>
__device__ __forceinline__ float didx(int j) { return j == N / 2 ? 0.0f : sidx<N>(j); }

// ---------------------------------------------------------------- phase A
__global__ void __launch_bounds__(64, 8) k_plasma(const float *__restrict__ nb, float *__restrict__ np, long long P, int Nxi, float q,
                         float c, float s, float ch, float sh) {
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= P) return;
    // two buffers of U cells of the line: the next U cells are in flight
    // while the current ones are marched (with one thread per transverse
    // point, 65,536 at N = 256, that keeps about 8 MB of loads outstanding)
    constexpr int U = 32;
    float n = 0.0f, d = 0.0f;
    float ba[U], bb[U];
    auto load = [&](float (&buf)[U], int j0) {
#pragma unroll
        for (int u = 0; u < U; ++u) buf[u] = (j0 + u < Nxi) ? __ldcg(nb + (long long)(j0 + u) * P + p) : 0.0f;
    };
    auto march = [&](const float (&buf)[U], int j0) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (j0 + u >= Nxi) break;
            const float rho = q * buf[u];
            const float un = n - rho;
            __stcg(np + (long long)(j0 + u) * P + p, fmaf(ch, un, fmaf(sh, d, rho)));
            const float x = fmaf(c, un, fmaf(s, d, rho));
            d = fmaf(-s, un, c * d);
            n = x;
        }
    };
    load(ba, 0);
    for (int j0 = 0; j0 < Nxi; j0 += 2 * U) {
        load(bb, j0 + U);
        march(ba, j0);
        load(ba, j0 + 2 * U);
        march(bb, j0 + U);
    }
}

// ---------------------------------------------------------------- K1
// grid (N / RB, Nxi); RB rows of one slice, packed in RB/2 complex rows.
template <int N, int RB>
__global__ void __launch_bounds__(256) k_rowfft(const float *__restrict__ np, float2 *__restrict__ S1) {
    extern __shared__ float2 sm[];
    float2 *tw = sm;
    float2 *A = sm + N / 2;
    float2 *B = A + (RB / 2) * N;
    constexpr int NH = N / 2 + 1;
    const long long slice = blockIdx.y;
    const int r0 = blockIdx.x * RB;
    make_twiddles<N>(tw);
    const float *src = np + slice * (long long)N * N;
    for (int i = threadIdx.x; i < (RB / 2) * N; i += blockDim.x) {
        const int pr = i / N, x = i - pr * N;
        A[i] = make_float2(src[(long long)(r0 + 2 * pr) * N + x], src[(long long)(r0 + 2 * pr + 1) * N + x]);
    }
    __syncthreads();
    float2 *R = fft_rows<N>(A, B, RB / 2, tw, false);
    float2 *dst = S1 + slice * (long long)N * NH;
    for (int i = threadIdx.x; i < (RB / 2) * NH; i += blockDim.x) {
        const int pr = i / NH, k = i - pr * NH;
        const float2 Z = R[pr * N + k], Zc = R[pr * N + ((N - k) & (N - 1))];
        // X1 = (Z + conj Zc)/2, X2 = (Z - conj Zc)/(2i)
        const float2 X1 = make_float2(0.5f * (Z.x + Zc.x), 0.5f * (Z.y - Zc.y));
        const float2 X2 = make_float2(0.5f * (Z.y + Zc.y), -0.5f * (Z.x - Zc.x));
        dst[(long long)(r0 + 2 * pr) * NH + k] = X1;
        dst[(long long)(r0 + 2 * pr + 1) * NH + k] = X2;
    }
}

// ---------------------------------------------------------------- K2
// grid (ceil(NH / CB), Nxi); CB spectral columns of one slice.
template <int N, int CB>
__global__ void __launch_bounds__(256) k_colfft(const float2 *__restrict__ S1, float2 *__restrict__ T1,
                                                float2 *__restrict__ T2, float ly, float lz) {
    extern __shared__ float2 sm[];
    constexpr int NH = N / 2 + 1;
    float2 *tw = sm;
    float2 *A = sm + N / 2;           // [2 CB][N]
    float2 *B = A + 2 * CB * N;       // [2 CB][N]
    const long long slice = blockIdx.y;
    const int c0 = blockIdx.x * CB;
    make_twiddles<N>(tw);
    const float2 *src = S1 + slice * (long long)N * NH;
    for (int i = threadIdx.x; i < CB * N; i += blockDim.x) {
        const int y = i / CB, c = i - y * CB;
        A[c * N + y] = (c0 + c < NH) ? src[(long long)y * NH + c0 + c] : make_float2(0.0f, 0.0f);
    }
    __syncthreads();
    float2 *R = fft_rows<N>(A, B, CB, tw, false);
    float2 *O = (R == A) ? B : A;     // free buffer for the two products
    const float inv = 1.0f / ((float)N * (float)N);
    const float ty = 6.283185307179586f / ly, tz = 6.283185307179586f / lz;
    for (int i = threadIdx.x; i < CB * N; i += blockDim.x) {
        const int c = i / N, jy = i - c * N;
        const int kzi = c0 + c;
        const float ky = ty * sidx<N>(jy), kz = tz * (float)(kzi == N / 2 ? -(N / 2) : kzi);
        const float kap = inv / (1.0f + ky * ky + kz * kz);
        const float2 X = R[c * N + jy];
        const float2 P = make_float2(kap * X.x, kap * X.y);
        const float kyd = ty * didx<N>(jy);
        O[c * N + jy] = P;                                        // Psi^
        O[(CB + c) * N + jy] = make_float2(-kyd * P.y, kyd * P.x); // i k_y Psi^
    }
    __syncthreads();
    float2 *Q = fft_rows<N>(O, R, 2 * CB, tw, true);
    float2 *d1 = T1 + slice * (long long)N * NH, *d2 = T2 + slice * (long long)N * NH;
    for (int i = threadIdx.x; i < CB * N; i += blockDim.x) {
        const int y = i / CB, c = i - y * CB;
        if (c0 + c < NH) {
            d1[(long long)y * NH + c0 + c] = Q[c * N + y];
            d2[(long long)y * NH + c0 + c] = Q[(CB + c) * N + y];
        }
    }
}

struct PushArgs {
    const float *np;
    float *nb, *G;
    const float *nb0, *gy, *gz;   // [N][N]
    float coef, h, dt, lz;
    int *err;
};

// ---------------------------------------------------------------- K3
// grid (N / RB, Nxi).  Rows r0 .. r0+RB-1: Z1_r = full(T1_r) + i full(i kz T1_r)
// (-> Psi, d_z Psi), Z2_pair = full(T2_r) + i full(T2_r+1) (-> d_y Psi).
template <int N, int RB>
__global__ void __launch_bounds__(256) k_rowinv_push(const float2 *__restrict__ T1, const float2 *__restrict__ T2,
                                                     const PushArgs a) {
    extern __shared__ float2 sm[];
    constexpr int NH = N / 2 + 1;
    constexpr int ROWS = RB + RB / 2;
    float2 *tw = sm;
    float2 *A = sm + N / 2;           // [ROWS][N]
    float2 *B = A + ROWS * N;
    const long long slice = blockIdx.y;
    const int r0 = blockIdx.x * RB;
    make_twiddles<N>(tw);
    const float2 *t1 = T1 + slice * (long long)N * NH, *t2 = T2 + slice * (long long)N * NH;
    const float tz = 6.283185307179586f / a.lz;
    for (int i = threadIdx.x; i < RB * N; i += blockDim.x) {
        const int r = i / N, k = i - r * N;
        const bool lo = k <= N / 2;
        const int kk = lo ? k : N - k;
        float2 X = t1[(long long)(r0 + r) * NH + kk];
        if (!lo) X.y = -X.y;
        const float kzd = tz * didx<N>(k);
        // X2 = i kzd X  ->  Z1 = X + i X2 = X - kzd X
        A[r * N + k] = make_float2(X.x - kzd * X.x, X.y - kzd * X.y);
    }
    for (int i = threadIdx.x; i < (RB / 2) * N; i += blockDim.x) {
        const int pr = i / N, k = i - pr * N;
        const bool lo = k <= N / 2;
        const int kk = lo ? k : N - k;
        float2 U = t2[(long long)(r0 + 2 * pr) * NH + kk], V = t2[(long long)(r0 + 2 * pr + 1) * NH + kk];
        if (!lo) { U.y = -U.y; V.y = -V.y; }
        A[(RB + pr) * N + k] = make_float2(U.x - V.y, U.y + V.x);   // U + i V
    }
    __syncthreads();
    float2 *R = fft_rows<N>(A, B, ROWS, tw, true);
    const long long base = slice * (long long)N * N;
    bool bad = false;
    for (int i = threadIdx.x; i < RB * N; i += blockDim.x) {
        const int r = i / N, z = i - r * N;
        const int y = r0 + r;
        const float2 Z1 = R[r * N + z];
        const float2 Z2 = R[(RB + r / 2) * N + z];
        const float psi = Z1.x, dz = Z1.y, dy = (r & 1) ? Z2.y : Z2.x;
        const long long o = base + (long long)y * N + z;
        const int t = y * N + z;
        const float S = a.coef * (a.nb0[t] * (psi - a.np[o]) + a.gy[t] * dy + a.gz[t] * dz);
        const float g = fmaf(a.h, S, a.G[o]);
        const float n = fmaf(a.dt, g, a.nb[o]);
        a.G[o] = g;
        a.nb[o] = n;
        bad |= !(fabsf(n) <= 3.0e38f) || !(fabsf(g) <= 3.0e38f);
    }
    if (bad) atomicOr(a.err, 1);
}

// K3 for N = 256: 128 threads = 8 teams, rows r0 .. r0 + 15 of one slice;
// team m owns rows y0 = r0 + 2m and y0 + 1 and needs nothing from the other
// teams' results: d_y Psi of both rows from one packed inverse transform of
// their T2 rows, then Psi and d_z Psi of each row from one of its T1 row.
// T1 and T2 are column-major ([xi][k_z][y]), so the block's 16 rows at one
// k_z are 128 contiguous bytes of each.  They are staged in shared memory as
// [T2, T1][k_z][8 pieces of two rows] (16-byte asynchronous copies, T2 and
// T1 in separate groups so that the d_y Psi transform starts while T1 is in
// flight; piece q of entry k sits at slot q ^ (k & 7), which spreads a
// team's reads over the banks).  The Hermitian extension reads entries k and
// 256 - k.  Once a team has read its T2 pieces, d_y Psi goes into those
// slots.  A transform leaves entry t + 16 k in thread t; the results are
// re-read so that the push runs on points 4 t + 64 i + c, whose operands the
// team loads and stores as 256 contiguous bytes per i, issued one transform
// ahead.  Shared memory is 52.6 KB per block, so four blocks fit on an SM.
// The block's 16-column strips of T2 and T1 (129 k_z rows of 128 bytes
// each) are staged by one thread as two tensor copies with the 128-byte
// swizzle: row k's 16-byte piece q lands at piece q ^ (k % 8) of the row,
// the layout the team reads, provided each strip starts on a 1024-byte
// boundary (T2 at row 0, T1 at row T1ROW = 136 of R).  The copies take no
// load/store-unit issue slots, which this kernel's shared-memory traffic
// keeps busy.  The maps view T1 / T2 as [n_xi * 129 rows][512 floats]; s0 is
// the launch's first slice.
constexpr int T1ROW = 136;
__global__ void __launch_bounds__(128, 4) k_rowinv_push256(const __grid_constant__ CUtensorMap tm1,
                                                           const __grid_constant__ CUtensorMap tm2, int s0,
                                                           const PushArgs a) {
    constexpr int N = 256, NH = 129, TSZ = 272;
    extern __shared__ __align__(1024) float2 sm_raw[];
    float2 *sm = reinterpret_cast<float2 *>(reinterpret_cast<unsigned char *>(sm_raw) +
                                            ((1024u - ((uint32_t)__cvta_generic_to_shared(sm_raw) & 1023u)) & 1023u));
    __shared__ __align__(8) uint64_t tbar[2];   // T2, T1 strips landed
    const long long slice = blockIdx.y;
    const int tm = threadIdx.x >> 4, t = threadIdx.x & 15;
    const int y0 = blockIdx.x * 16 + 2 * tm;
    float2 *R = sm;                                 // [T2 rows 0..128, T1 rows T1ROW..][16 columns]
    float2 *tw = sm + (T1ROW + NH) * 16, *Ts = tw + TWN + tm * TSZ;
    if (threadIdx.x == 0) {
        const uint32_t b0 = (uint32_t)__cvta_generic_to_shared(&tbar[0]), b1 = (uint32_t)__cvta_generic_to_shared(&tbar[1]);
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b0));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        const int x = blockIdx.x * 32, y = (s0 + (int)slice) * NH;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint32_t b = h ? b1 : b0;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(NH * 128) : "memory");
            asm volatile(
                "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
                ::"r"((uint32_t)__cvta_generic_to_shared(R + (h ? T1ROW : 0) * 16)),
                "l"(reinterpret_cast<uint64_t>(h ? &tm1 : &tm2)), "r"(x), "r"(y), "r"(b) : "memory");
        }
    }
    // bounded wait on a strip (every thread); false: it did not land
    auto strip_wait = [&](int h) {
        const uint32_t b = (uint32_t)__cvta_generic_to_shared(&tbar[h]);
        uint32_t done = 0;
        for (long long spin = 0; spin < (1LL << 24) && !done; ++spin)
            asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0; selp.u32 %0, 1, 0, p; }"
                         : "=r"(done) : "r"(b) : "memory");
        return done != 0;
    };
    // a strip that did not land in time: wait once more (bounded) and report it
    auto strip = [&](int h) {
        if (!strip_wait(h)) {
            strip_wait(h);
            atomicOr(a.err, 2);
        }
    };
    const long long base = slice * (long long)N * N;
    const float tz = 6.283185307179586f / a.lz;
    float4 lnp[4], lnb[4], lg[4];
    auto issue = [&](int rr) {
        const long long o = base + (long long)(y0 + rr) * N;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int z = 4 * t + 64 * i;
            lnp[i] = __ldcg(reinterpret_cast<const float4 *>(a.np + o + z));
            lnb[i] = __ldcg(reinterpret_cast<const float4 *>(a.nb + o + z));
            lg[i] = __ldcg(reinterpret_cast<const float4 *>(a.G + o + z));
        }
    };
    issue(0);
    make_tw256_p2(tw);
    __syncthreads();   // twiddles; the strip barriers initialised
    strip(0);   // the staged T2 strip
    // entry k = t + 16 m of a row's Hermitian extension: entry kk of the half
    // spectrum, conjugated past 128
    float2 x[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        const int k = t + 16 * m, kk = k <= 128 ? k : N - k;
        const float4 uv = *reinterpret_cast<const float4 *>(R + kk * 16 + 2 * (tm ^ (kk & 7)));   // rows y0, y0 + 1 of T2
        float2 U = make_float2(uv.x, uv.y), V = make_float2(uv.z, uv.w);
        if (k > 128) { U.y = -U.y; V.y = -V.y; }
        x[m] = make_float2(U.x - V.y, U.y + V.x);   // U + i V
    }
    fft256_reg<true, true>(x, Ts, tw, t);
    // entry z of the row pair's d_y Psi goes to this team's slot of entry
    // u / 2, half u % 2, u = (z & ~15) | ((z & 15) ^ ((z / 16) & 3)): the
    // stores (z = t + 16 k) and the push's loads (z = 4 t + 64 i + c) each
    // touch 16 distinct bank pairs
    auto dslot = [&](int z) {
        const int u = (z & ~15) | ((z & 15) ^ ((z >> 4) & 3)), k = u >> 1;
        return k * 16 + 2 * (tm ^ (k & 7)) + (u & 1);
    };
#pragma unroll
    for (int k2 = 0; k2 < 16; ++k2) R[dslot(t + 16 * k2)] = x[k2];
    strip(1);   // the staged T1 strip
    __syncthreads();
    bool bad = false;
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
        // Psi + i d_z Psi = inverse transform of X - k_z X (X the Hermitian extension of the T1 row)
#pragma unroll
        for (int m = 0; m < 16; ++m) {
            const int k = t + 16 * m, kk = k <= 128 ? k : N - k;
            float2 X = R[(T1ROW + kk) * 16 + 2 * (tm ^ (kk & 7)) + rr];
            if (k > 128) X.y = -X.y;
            const float kzd = tz * (k == 128 ? 0.0f : (float)(k < 128 ? k : k - 256));
            x[m] = make_float2(X.x - kzd * X.x, X.y - kzd * X.y);
        }
        fft256_reg<true, true>(x, Ts, tw, t);
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) Ts[t * 17 + k2] = x[k2];
        __syncwarp();
        const long long o = base + (long long)(y0 + rr) * N;
        const int q = (y0 + rr) * N;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int z = 4 * t + 64 * i;
            const float4 n0v = __ldg(reinterpret_cast<const float4 *>(a.nb0 + q + z));
            const float4 gyv4 = __ldg(reinterpret_cast<const float4 *>(a.gy + q + z));
            const float4 gzv4 = __ldg(reinterpret_cast<const float4 *>(a.gz + q + z));
            float e[4], f[4];
            const float npa[4] = {lnp[i].x, lnp[i].y, lnp[i].z, lnp[i].w}, nbv[4] = {lnb[i].x, lnb[i].y, lnb[i].z, lnb[i].w};
            const float gv[4] = {lg[i].x, lg[i].y, lg[i].z, lg[i].w}, n0[4] = {n0v.x, n0v.y, n0v.z, n0v.w};
            const float gyv[4] = {gyv4.x, gyv4.y, gyv4.z, gyv4.w}, gzv[4] = {gzv4.x, gzv4.y, gzv4.z, gzv4.w};
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                // point z + c: (z + c) % 16 = 4 (t % 4) + c, (z + c) / 16 = t / 4 + 4 i
                const float2 pz = Ts[(4 * (t & 3) + c) * 17 + (t >> 2) + 4 * i];
                const float2 dyp = R[dslot(z + c)];
                const float dyv = rr ? dyp.y : dyp.x;
                const float S = a.coef * (n0[c] * (pz.x - npa[c]) + gyv[c] * dyv + gzv[c] * pz.y);
                f[c] = fmaf(a.h, S, gv[c]);
                e[c] = fmaf(a.dt, f[c], nbv[c]);
                bad |= !(fabsf(e[c]) <= 3.0e38f) || !(fabsf(f[c]) <= 3.0e38f);
            }
            __stcg(reinterpret_cast<float4 *>(a.G + o + z), make_float4(f[0], f[1], f[2], f[3]));
            __stcg(reinterpret_cast<float4 *>(a.nb + o + z), make_float4(e[0], e[1], e[2], e[3]));
        }
        __syncwarp();   // Ts is reused by the next transform
        if (rr == 0) issue(1);
    }
    if (bad) atomicOr(a.err, 1);
}

// Philox4x32-10 (Salmon et al., SC'11) and the seed: n_b = A (n_b0/peak) g +
// base(y, z), G = 0; g a standard normal per (cell, point) or a user field.
__device__ __forceinline__ void philox(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
        const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
        k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
    }
}

__global__ void k_seed(float *nb, float *G, long long P, int Nxi, const float *nb0, const float *base, float amp_rel,
                       uint64_t seed, const float *user) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= P * Nxi) return;
    const long long p = i % P;
    const int j = (int)(i / P);
    double g;
    if (user) {
        g = user[i];
    } else {
        uint32_t c[4] = {(uint32_t)j, (uint32_t)p, 0x52324E53u, 0u};
        philox(c, (uint32_t)seed, (uint32_t)(seed >> 32));
        const uint64_t m1 = ((uint64_t)c[0] << 21) | (c[1] >> 11);
        const uint64_t m2 = ((uint64_t)c[2] << 21) | (c[3] >> 11);
        const double u1 = ((double)m1 + 0.5) * 0x1.0p-53, u2 = ((double)m2 + 0.5) * 0x1.0p-53;
        g = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
    }
    nb[i] = (float)((double)amp_rel * nb0[p] * g + base[p]);
    G[i] = 0.0f;
}

}  // namespace r2

struct qs_r2 {
    qs_r2_params p{};
    int N = 0;
    long long P = 0, cells = 0;
    cudaStream_t stream = nullptr;
    qs_allocator alloc{};
    bool has_alloc = false;
    std::vector<void *> bufs;
    float *nb = nullptr, *G = nullptr, *np = nullptr, *nb0 = nullptr, *gy = nullptr, *gz = nullptr, *base = nullptr;
    float2 *S1 = nullptr, *T1 = nullptr, *T2 = nullptr;
    CUtensorMap tmT1{}, tmT2{};          // N = 256: T1 / T2 as [n_xi * 129][512] floats (the push kernel's strips)
    int *err = nullptr;
    long long step = 0;
    long long launches = 0;
};

namespace {

constexpr int RB = 16, CB = 16;

template <int N>
size_t smem_k1() { return sizeof(float2) * (N / 2 + 2 * (RB / 2) * N); }
template <int N>
size_t smem_k2() { return sizeof(float2) * (N / 2 + 4 * CB * N); }
template <int N>
size_t smem_k3() { return sizeof(float2) * (N / 2 + 2 * (RB + RB / 2) * N); }

// T1 or T2 (n_xi slices of [129 k_z][256 y] float2) as a 2-D tensor of
// floats, [n_xi * 129 rows][512], for the push kernel's strips: boxes of 32
// floats (16 columns, 128 bytes) x 129 rows with the 128-byte swizzle
bool r2_tmap(CUtensorMap *tm, float2 *T, long long n_xi) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
            return false;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const cuuint64_t dims[2] = {512u, (cuuint64_t)n_xi * 129};
    const cuuint64_t strides[1] = {512u * 4};
    const cuuint32_t box[2] = {32u, 129u};
    const cuuint32_t es[2] = {1, 1};
    return encode(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, T, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

constexpr size_t SMEM_K1_256 = sizeof(float2) * (r2::TWN + 16 * 274);
constexpr size_t SMEM_K2_256 = sizeof(float2) * (r2::TWN + 8 * 272);
constexpr size_t SMEM_K3_256 = 1024 + sizeof(float2) * ((r2::T1ROW + 129) * 16 + r2::TWN + 8 * 272);   // + alignment slack

template <int N>
cudaError_t set_attrs() {
    if constexpr (N == 256) {
        cudaError_t e = cudaFuncSetAttribute(r2::k_rowfft256, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_K1_256);
        if (!e) e = cudaFuncSetAttribute(r2::k_colfft256, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_K2_256);
        if (!e) e = cudaFuncSetAttribute(r2::k_rowinv_push256, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_K3_256);
        return e;
    }
    cudaError_t e = cudaFuncSetAttribute(r2::k_rowfft<N, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_k1<N>());
    if (!e) e = cudaFuncSetAttribute(r2::k_colfft<N, CB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_k2<N>());
    if (!e) e = cudaFuncSetAttribute(r2::k_rowinv_push<N, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_k3<N>());
    return e;
}

template <int N>
cudaError_t step_n(qs_r2 *c, float h) {
    const qs_r2_params &p = c->p;
    const double D = p.dxi;
    const float q = (float)p.species.q;
    r2::k_plasma<<<(unsigned)((c->P + 63) / 64), 64, 0, c->stream>>>(
        c->nb, c->np, c->P, p.n_xi, q, (float)std::cos(D), (float)std::sin(D), (float)std::cos(0.5 * D),
        (float)std::sin(0.5 * D));
    constexpr int NH = N / 2 + 1;
    r2::PushArgs a{c->np, c->nb, c->G, c->nb0, c->gy, c->gz,
                   (float)(-p.species.q / (p.species.m * p.gamma_b)), h, (float)p.dt, (float)p.L_perp, c->err};
    c->launches += 1;
    // the transform kernels take the slice from blockIdx.y (at most 65,535
    // per launch): longer lines go in chunks, with the slice-major arrays
    // offset to the chunk's first slice.  QS_R2_CHUNK sets a smaller chunk
    // (tests: the chunked launches at sizes an oracle can check)
    long long MAXY = 65535;
    if (const char *v = getenv("QS_R2_CHUNK")) {
        const long long k = atoll(v);
        if (k >= 1 && k < MAXY) MAXY = k;
    }
    for (long long s0 = 0; s0 < p.n_xi; s0 += MAXY) {
        const unsigned ns = (unsigned)std::min<long long>(MAXY, p.n_xi - s0);
        const long long po = s0 * c->P, so = s0 * (long long)N * NH;
        r2::PushArgs as = a;
        as.np += po; as.nb += po; as.G += po;
        if constexpr (N == 256) {
            r2::k_rowfft256<<<dim3(256 / 32, ns), 256, SMEM_K1_256, c->stream>>>(c->np + po, c->S1 + so);
            r2::k_colfft256<<<dim3(16, ns), 128, SMEM_K2_256, c->stream>>>(
                c->S1 + so, c->T1 + so, c->T2 + so, (float)p.L_perp, (float)p.L_perp);
            r2::k_rowinv_push256<<<dim3(256 / 16, ns), 128, SMEM_K3_256, c->stream>>>(c->tmT1, c->tmT2, (int)s0, as);
        } else {
            r2::k_rowfft<N, RB><<<dim3(N / RB, ns), 256, smem_k1<N>(), c->stream>>>(c->np + po, c->S1 + so);
            r2::k_colfft<N, CB><<<dim3((NH + CB - 1) / CB, ns), 256, smem_k2<N>(), c->stream>>>(
                c->S1 + so, c->T1 + so, c->T2 + so, (float)p.L_perp, (float)p.L_perp);
            r2::k_rowinv_push<N, RB><<<dim3(N / RB, ns), 256, smem_k3<N>(), c->stream>>>(c->T1 + so, c->T2 + so, as);
        }
        c->launches += 3;
    }
    return cudaGetLastError();
}

qs_status r2_alloc(qs_r2 *c, size_t bytes, void **out) {
    void *p = nullptr;
    if (c->has_alloc) {
        p = c->alloc.alloc(bytes, c->alloc.user);
        if (!p) return QS_ERR_OOM;
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return QS_ERR_OOM;
    }
    c->bufs.push_back(p);
    *out = p;
    return QS_OK;
}

template <typename T>
qs_status r2_alloc_t(qs_r2 *c, size_t bytes, T **out) {
    void *v = nullptr;
    qs_status s = r2_alloc(c, bytes, &v);
    *out = static_cast<T *>(v);
    return s;
}

}  // namespace

extern "C" {

qs_status qs_r2_init(const qs_r2_params *p, const qs_allocator *alloc, void *stream, qs_r2 **out) {
    QS_RANGE("qs_r2_init");
    if (!p || !out) return QS_ERR_ARG;
    *out = nullptr;
    const int N = p->n_perp;
    if (!(N == 32 || N == 64 || N == 128 || N == 256)) return QS_ERR_UNSUPPORTED;
    if (p->n_xi < 1 || !(p->dxi > 0) || !(p->dt > 0) || !(p->gamma_b > 1) || !(p->L_perp > 0) ||
        !(p->species.m > 0) || !(p->species.density_ratio > 0) || (!p->uniform && !(p->sigma_r > 0)))
        return QS_ERR_ARG;
    qs_r2 *c = new qs_r2();
    c->p = *p;
    c->N = N;
    c->P = (long long)N * N;
    c->cells = c->P * p->n_xi;
    c->stream = static_cast<cudaStream_t>(stream);
    if (alloc && alloc->alloc && alloc->free) { c->alloc = *alloc; c->has_alloc = true; }
    const long long NH = N / 2 + 1;
    const size_t spec = sizeof(float2) * (size_t)p->n_xi * N * NH;
    qs_status s;
    if ((s = r2_alloc_t(c, sizeof(float) * c->cells, &c->nb)) || (s = r2_alloc_t(c, sizeof(float) * c->cells, &c->G)) ||
        (s = r2_alloc_t(c, sizeof(float) * c->cells, &c->np)) || (s = r2_alloc_t(c, spec, &c->S1)) ||
        (s = r2_alloc_t(c, spec, &c->T1)) || (s = r2_alloc_t(c, spec, &c->T2)) ||
        (s = r2_alloc_t(c, sizeof(float) * c->P * 4, &c->nb0)) || (s = r2_alloc_t(c, sizeof(int) * 4, &c->err))) {
        qs_r2_free(c);
        return s;
    }
    if (N == 256 && (!r2_tmap(&c->tmT1, c->T1, p->n_xi) || !r2_tmap(&c->tmT2, c->T2, p->n_xi))) {
        qs_r2_free(c);
        return QS_ERR_CUDA;
    }
    c->gy = c->nb0 + c->P;
    c->gz = c->nb0 + 2 * c->P;
    c->base = c->nb0 + 3 * c->P;
    // transverse profile and its analytic gradient at cell centres (FP64 -> FP32)
    std::vector<float> t(4 * c->P);
    const double d = p->L_perp / N, s2 = p->sigma_r * p->sigma_r, dens = p->species.density_ratio;
    for (int iy = 0; iy < N; ++iy)
        for (int iz = 0; iz < N; ++iz) {
            const double y = (iy + 0.5) * d - 0.5 * p->L_perp, z = (iz + 0.5) * d - 0.5 * p->L_perp;
            const double n0 = p->uniform ? dens : dens * std::exp(-(y * y + z * z) / (2 * s2));
            const long long k = (long long)iy * N + iz;
            t[k] = (float)n0;
            t[c->P + k] = p->uniform ? 0.0f : (float)(-(y / s2) * n0);
            t[2 * c->P + k] = p->uniform ? 0.0f : (float)(-(z / s2) * n0);
            t[3 * c->P + k] = 0.0f;
        }
    // all on the context's stream, then one wait for it (the host vector t
    // must outlive the copy; the stream may be one that does not synchronise
    // with the legacy default stream)
    cudaError_t e = cudaMemcpyAsync(c->nb0, t.data(), sizeof(float) * t.size(), cudaMemcpyHostToDevice, c->stream);
    if (!e) e = cudaMemsetAsync(c->err, 0, sizeof(int) * 4, c->stream);
    if (!e) e = cudaMemsetAsync(c->nb, 0, sizeof(float) * c->cells, c->stream);
    if (!e) e = cudaMemsetAsync(c->G, 0, sizeof(float) * c->cells, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    if (!e) e = N == 32 ? set_attrs<32>() : N == 64 ? set_attrs<64>() : N == 128 ? set_attrs<128>() : set_attrs<256>();
    if (e) { cudaGetLastError(); qs_r2_free(c); return QS_ERR_CUDA; }
    *out = c;
    return QS_OK;
}

qs_status qs_r2_seed(qs_r2 *c, uint64_t seed, double amplitude, double centroid_offset, const float *user,
                     size_t user_bytes, int user_on_host) {
    QS_RANGE("qs_r2_seed");
    if (!c) return QS_ERR_ARG;
    const qs_r2_params &p = c->p;
    const int N = c->N;
    // base(y, z) = n_b0(y - offset, z) - n_b0(y, z): exact shifted-profile seed
    std::vector<float> b(c->P, 0.0f);
    if (centroid_offset != 0.0 && !p.uniform) {
        const double d = p.L_perp / N, s2 = p.sigma_r * p.sigma_r, dens = p.species.density_ratio;
        for (int iy = 0; iy < N; ++iy)
            for (int iz = 0; iz < N; ++iz) {
                const double y = (iy + 0.5) * d - 0.5 * p.L_perp, z = (iz + 0.5) * d - 0.5 * p.L_perp;
                const double sh = dens * std::exp(-((y - centroid_offset) * (y - centroid_offset) + z * z) / (2 * s2));
                const double n0 = dens * std::exp(-(y * y + z * z) / (2 * s2));
                b[(long long)iy * N + iz] = (float)(sh - n0);
            }
    }
    cudaError_t e = cudaMemcpyAsync(c->base, b.data(), sizeof(float) * c->P, cudaMemcpyHostToDevice, c->stream);
    const float *u = nullptr;
    void *tmp = nullptr;
    if (user) {
        if (user_bytes < sizeof(float) * (size_t)c->cells) return QS_ERR_ARG;
        if (user_on_host) {
            if (r2_alloc(c, sizeof(float) * c->cells, &tmp)) return QS_ERR_OOM;
            if (!e) e = cudaMemcpyAsync(tmp, user, sizeof(float) * c->cells, cudaMemcpyHostToDevice, c->stream);
            u = static_cast<const float *>(tmp);
        } else {
            u = user;
        }
    }
    if (!e) {
        r2::k_seed<<<(unsigned)((c->cells + 255) / 256), 256, 0, c->stream>>>(
            c->nb, c->G, c->P, p.n_xi, c->nb0, c->base, (float)(amplitude / p.species.density_ratio), seed, u);
        e = cudaGetLastError();
    }
    if (!e) e = cudaMemsetAsync(c->err, 0, sizeof(int) * 4, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);   // host tables and staging die here
    if (tmp) {
        if (c->has_alloc) c->alloc.free(tmp, c->alloc.user); else cudaFree(tmp);
        c->bufs.pop_back();
    }
    c->step = 0;
    return e ? QS_ERR_CUDA : QS_OK;
}

qs_status qs_r2_step(qs_r2 *c, int n_steps) {
    QS_RANGE("qs_r2_step");
    if (!c || n_steps < 1) return QS_ERR_ARG;
    for (int i = 0; i < n_steps; ++i) {
        const float h = (float)(c->step == 0 ? 0.5 * c->p.dt : c->p.dt);
        cudaError_t e;
        switch (c->N) {
        case 32: e = step_n<32>(c, h); break;
        case 64: e = step_n<64>(c, h); break;
        case 128: e = step_n<128>(c, h); break;
        default: e = step_n<256>(c, h); break;
        }
        if (e) return QS_ERR_CUDA;
        ++c->step;
    }
    return QS_OK;
}

qs_status qs_r2_read(qs_r2 *c, int what, float *out, size_t out_bytes, int on_host) {
    if (!c || !out || what < 0 || what > 2 || out_bytes < sizeof(float) * (size_t)c->cells) return QS_ERR_ARG;
    const float *src = what == 0 ? c->nb : what == 1 ? c->G : c->np;
    cudaError_t e = cudaMemcpyAsync(out, src, sizeof(float) * c->cells,
                                    on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, c->stream);
    if (!e && on_host) e = cudaStreamSynchronize(c->stream);
    return e ? QS_ERR_CUDA : QS_OK;
}

qs_status qs_r2_sync(qs_r2 *c) {
    if (!c) return QS_ERR_ARG;
    int e = 0;
    // on the context's stream (a plain cudaMemcpy would wait for every blocking stream)
    if (cudaMemcpyAsync(&e, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
        return QS_ERR_CUDA;
    return e ? QS_ERR_NONFINITE : QS_OK;
}

int64_t qs_r2_launch_count(const qs_r2 *c) { return c ? c->launches : -1; }

void qs_r2_free(qs_r2 *c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream); else cudaDeviceSynchronize();
    for (void *p : c->bufs) {
        if (c->has_alloc) c->alloc.free(p, c->alloc.user); else cudaFree(p);
    }
    delete c;
}

}  // extern "C"
