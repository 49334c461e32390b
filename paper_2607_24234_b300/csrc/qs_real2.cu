// qs_real2.cu -- finite-width beam on a periodic transverse grid (sm_103a).
//
// Narrow beams (Sec. IV.B: self-modulation and hosing) need the transverse
// profile n_b0(y, z) in real space.  Per slow-time step:
//   A. plasma response per transverse point, (d_xi^2 + 1) n_p = q n_b
//      (Eq. 5, local in r_perp): one thread per point marches xi with the
//      exact cell propagator and writes n_p at the cell centres;
//   B. per xi slice, the screened Poisson solve of Eq. (14),
//      Psi^ = n_p^ / (1 + k^2), and grad_perp Psi by spectral derivatives,
//      with hand-written radix-2 Stockham FFTs in shared memory:
//        K1  row FFTs along z (two real rows packed per complex FFT) ->
//            half spectrum S1 [xi][y][N/2+1];
//        K2  column FFTs along y, multiply by kappa and i k_y kappa, two
//            inverse column FFTs -> T1 = Psi~, T2 = (d_y Psi)~ [xi][y][N/2+1];
//        K3  inverse row FFTs (Psi and d_z Psi packed as real/imag of one
//            FFT, d_y Psi of two rows packed in another) fused with the push
//            d_tau G = -(q/(m gamma)) [n_b0 (Psi - n_p) + grad n_b0 . grad Psi],
//            n_b += dt G (kick-drift leapfrog, first kick dt/2).
// The gamma^-3 term is dropped here (gamma_b >> 1 for narrow-beam cases).
// State and intermediates are FP32, laid out [xi][y][z] with z fastest.
#include <cuda_runtime.h>

#include <cmath>
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
// 16-point DFT is radix 4 x 4.  tw256[j] = exp(-2 pi i j / 256).
// ---------------------------------------------------------------------------
template <bool INV>
__device__ __forceinline__ void dft4(float2 &a0, float2 &a1, float2 &a2, float2 &a3) {
    const float2 t0 = make_float2(a0.x + a2.x, a0.y + a2.y), t1 = make_float2(a0.x - a2.x, a0.y - a2.y);
    const float2 t2 = make_float2(a1.x + a3.x, a1.y + a3.y), t3 = make_float2(a1.x - a3.x, a1.y - a3.y);
    const float2 m3 = make_float2(t3.y, -t3.x);   // -i t3
    a0 = make_float2(t0.x + t2.x, t0.y + t2.y);
    a2 = make_float2(t0.x - t2.x, t0.y - t2.y);
    if (INV) {
        a1 = make_float2(t1.x - m3.x, t1.y - m3.y);
        a3 = make_float2(t1.x + m3.x, t1.y + m3.y);
    } else {
        a1 = make_float2(t1.x + m3.x, t1.y + m3.y);
        a3 = make_float2(t1.x - m3.x, t1.y - m3.y);
    }
}

template <bool INV>
__device__ __forceinline__ float2 twid(const float2 *tw256, int j) {
    float2 w = tw256[j & 255];
    if (INV) w.y = -w.y;
    return w;
}

// x[k] <- sum_m x[m] W16^(m k) (conjugate twiddles when INV)
template <bool INV>
__device__ __forceinline__ void dft16(float2 (&x)[16], const float2 *tw256) {
    float2 y[16];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        float2 a0 = x[b], a1 = x[4 + b], a2 = x[8 + b], a3 = x[12 + b];
        dft4<INV>(a0, a1, a2, a3);
        y[4 * b + 0] = a0;
        y[4 * b + 1] = cmul(a1, twid<INV>(tw256, 16 * b));
        y[4 * b + 2] = cmul(a2, twid<INV>(tw256, 32 * b));
        y[4 * b + 3] = cmul(a3, twid<INV>(tw256, 48 * b));
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        float2 a0 = y[c], a1 = y[4 + c], a2 = y[8 + c], a3 = y[12 + c];
        dft4<INV>(a0, a1, a2, a3);
        x[c] = a0; x[c + 4] = a1; x[c + 8] = a2; x[c + 12] = a3;
    }
}

// in-place FFT of one 256-entry row in shared memory by a 16-thread team;
// every thread of the warp must call it (both half-warp teams in step)
template <bool INV>
__device__ __forceinline__ void fft256_team(float2 *row, float2 *T, const float2 *tw256, int t) {
    float2 x[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) x[m] = row[t + 16 * m];
    dft16<INV>(x, tw256);
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) T[k1 * 17 + t] = cmul(x[k1], twid<INV>(tw256, t * k1));
    __syncwarp();
#pragma unroll
    for (int tt = 0; tt < 16; ++tt) x[tt] = T[t * 17 + tt];
    dft16<INV>(x, tw256);
#pragma unroll
    for (int k2 = 0; k2 < 16; ++k2) row[t + 16 * k2] = x[k2];
    __syncwarp();
}

__device__ __forceinline__ void make_tw256(float2 *tw) {
    for (int j = threadIdx.x; j < 256; j += blockDim.x) {
        float s, c;
        sincospif(-2.0f * j / 256.0f, &s, &c);
        tw[j] = make_float2(c, s);
    }
}

// K1 for N = 256: 32 rows (16 packed) per CTA, 16 teams
__global__ void __launch_bounds__(256) k_rowfft256(const float *__restrict__ np, float2 *__restrict__ S1) {
    constexpr int N = 256, NH = 129, PR = 16;
    extern __shared__ float2 sm[];
    float2 *tw = sm, *A = sm + 256, *T = A + PR * N;
    const long long slice = blockIdx.y;
    const int r0 = blockIdx.x * 2 * PR;
    const int team = threadIdx.x >> 4, t = threadIdx.x & 15;
    make_tw256(tw);
    const float *src = np + slice * (long long)N * N;
    // 4-byte asynchronous copies of the two real rows into the (re, im)
    // halves of each packed complex row, all in flight at once
    for (int i = threadIdx.x; i < PR * N; i += blockDim.x) {
        const int pr = i >> 8, x = i & 255;
        const uint32_t d = (uint32_t)__cvta_generic_to_shared(A + i);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src + (long long)(r0 + 2 * pr) * N + x)
                     : "memory");
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d + 4u), "l"(src + (long long)(r0 + 2 * pr + 1) * N + x)
                     : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    fft256_team<false>(A + team * N, T + team * 272, tw, t);
    __syncthreads();
    float2 *dst = S1 + slice * (long long)N * NH;
    for (int i = threadIdx.x; i < PR * NH; i += blockDim.x) {
        const int pr = i / NH, k = i - pr * NH;
        const float2 Z = A[pr * N + k], Zc = A[pr * N + ((N - k) & (N - 1))];
        dst[(long long)(r0 + 2 * pr) * NH + k] = make_float2(0.5f * (Z.x + Zc.x), 0.5f * (Z.y - Zc.y));
        dst[(long long)(r0 + 2 * pr + 1) * NH + k] = make_float2(0.5f * (Z.y + Zc.y), -0.5f * (Z.x - Zc.x));
    }
}

// K2 for N = 256: 16 spectral columns per CTA, one team per column
__global__ void __launch_bounds__(256) k_colfft256(const float2 *__restrict__ S1, float2 *__restrict__ T1,
                                                   float2 *__restrict__ T2, float ly, float lz) {
    constexpr int N = 256, NH = 129, CBn = 16, LD = N + 1;   // padded column stride
    extern __shared__ float2 sm[];
    float2 *tw = sm, *A = sm + 256, *A2 = A + CBn * LD, *T = A2 + CBn * LD;
    const long long slice = blockIdx.y;
    const int c0 = blockIdx.x * CBn;
    const int team = threadIdx.x >> 4, t = threadIdx.x & 15;
    make_tw256(tw);
    const float2 *src = S1 + slice * (long long)N * NH;
    // 8-byte asynchronous copies, all in flight at once (zero fill past the
    // last spectral column)
    for (int i = threadIdx.x; i < CBn * N; i += blockDim.x) {
        const int y = i >> 4, c = i & 15;
        const bool in = c0 + c < NH;
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(A + c * LD + y)),
                     "l"(src + (in ? (long long)y * NH + c0 + c : 0)), "r"(in ? 8 : 0) : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    float2 *col = A + team * LD, *col2 = A2 + team * LD;
    fft256_team<false>(col, T + team * 272, tw, t);
    const int kzi = c0 + team;
    const float inv = 1.0f / (256.0f * 256.0f);
    const float ty = 6.283185307179586f / ly, tz = 6.283185307179586f / lz;
    const float kz = tz * (float)(kzi == 128 ? -128 : kzi);
#pragma unroll 4
    for (int m = 0; m < 16; ++m) {
        const int jy = t + 16 * m;
        const float sy = (float)(jy < 128 ? jy : jy - 256);
        const float ky = ty * sy, kyd = jy == 128 ? 0.0f : ky;
        const float kap = inv / (1.0f + ky * ky + kz * kz);
        const float2 X = col[jy];
        const float2 P = make_float2(kap * X.x, kap * X.y);
        col[jy] = P;
        col2[jy] = make_float2(-kyd * P.y, kyd * P.x);
    }
    __syncwarp();
    fft256_team<true>(col, T + team * 272, tw, t);
    fft256_team<true>(col2, T + team * 272, tw, t);
    __syncthreads();
    float2 *d1 = T1 + slice * (long long)N * NH, *d2 = T2 + slice * (long long)N * NH;
    for (int i = threadIdx.x; i < CBn * N; i += blockDim.x) {
        const int y = i >> 4, c = i & 15;
        if (c0 + c < NH) {
            __stcg(d1 + (long long)y * NH + c0 + c, A[c * LD + y]);
            __stcg(d2 + (long long)y * NH + c0 + c, A2[c * LD + y]);
        }
    }
}

// signed spectral index and its derivative version (Nyquist zeroed)
template <int N>
__device__ __forceinline__ float sidx(int j) { return (float)(j < N / 2 ? j : j - N); }
template <int N>
__device__ __forceinline__ float didx(int j) { return j == N / 2 ? 0.0f : sidx<N>(j); }

// ---------------------------------------------------------------- phase A
__global__ void k_plasma(const float *__restrict__ nb, float *__restrict__ np, long long P, int Nxi, float q,
                         float c, float s, float ch, float sh) {
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= P) return;
    constexpr int U = 8;
    float n = 0.0f, d = 0.0f;
    float buf[U];
    for (int j0 = 0; j0 < Nxi; j0 += U) {
#pragma unroll
        for (int u = 0; u < U; ++u)
            buf[u] = (j0 + u < Nxi) ? __ldcg(nb + (long long)(j0 + u) * P + p) : 0.0f;
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

// K3 for N = 256: 16 rows per CTA -> 16 Z1 rows + 8 Z2 rows; teams 0..7
// transform two rows, teams 8..15 one (uniform within each warp).
__global__ void __launch_bounds__(256) k_rowinv_push256(const float2 *__restrict__ T1, const float2 *__restrict__ T2,
                                                        const PushArgs a) {
    constexpr int N = 256, NH = 129, RBn = 16;
    extern __shared__ float2 sm[];
    float2 *tw = sm, *A = sm + 256, *T = A + (RBn + RBn / 2) * N;
    const long long slice = blockIdx.y;
    const int r0 = blockIdx.x * RBn;
    const int team = threadIdx.x >> 4, t = threadIdx.x & 15;
    make_tw256(tw);
    // issue the push operands' loads first: they land while the transforms run
    const long long base = slice * (long long)N * N;
    constexpr int PER = RBn * N / 256;          // 16 elements per thread
    float pnp[PER], pnb[PER], pg[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int i = threadIdx.x + u * 256;
        const long long o = base + (long long)(r0 + (i >> 8)) * N + (i & 255);
        pnp[u] = __ldcg(a.np + o);
        pnb[u] = __ldcg(a.nb + o);
        pg[u] = __ldcg(a.G + o);
    }
    const float2 *t1 = T1 + slice * (long long)N * NH, *t2 = T2 + slice * (long long)N * NH;
    const float tz = 6.283185307179586f / a.lz;
    // stage the raw half spectra of the CTA's rows (T1 and T2, RBn rows each)
    // in the FFT scratch with 8-byte asynchronous copies, all in flight at once
    float2 *S1s = T, *S2s = T + RBn * NH;        // 2 RBn NH <= 16 * 272 entries
    for (int i = threadIdx.x; i < RBn * NH; i += blockDim.x) {
        const int r = i / NH, k = i - r * NH;
        const long long o = (long long)(r0 + r) * NH + k;
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(S1s + i)),
                     "l"(t1 + o) : "memory");
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(S2s + i)),
                     "l"(t2 + o) : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    for (int i = threadIdx.x; i < RBn * N; i += blockDim.x) {
        const int r = i >> 8, k = i & 255;
        const bool lo = k <= 128;
        const int kk = lo ? k : N - k;
        float2 X = S1s[r * NH + kk];
        if (!lo) X.y = -X.y;
        const float kzd = tz * (k == 128 ? 0.0f : (float)(k < 128 ? k : k - 256));
        A[r * N + k] = make_float2(X.x - kzd * X.x, X.y - kzd * X.y);
    }
    for (int i = threadIdx.x; i < (RBn / 2) * N; i += blockDim.x) {
        const int pr = i >> 8, k = i & 255;
        const bool lo = k <= 128;
        const int kk = lo ? k : N - k;
        float2 U = S2s[(2 * pr) * NH + kk], V = S2s[(2 * pr + 1) * NH + kk];
        if (!lo) { U.y = -U.y; V.y = -V.y; }
        A[(RBn + pr) * N + k] = make_float2(U.x - V.y, U.y + V.x);
    }
    __syncthreads();   // the FFTs below reuse the scratch
    fft256_team<true>(A + team * N, T + team * 272, tw, t);
    if (team < 8) fft256_team<true>(A + (RBn + team) * N, T + team * 272, tw, t);
    __syncthreads();
    bool bad = false;
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int i = threadIdx.x + u * 256;
        const int r = i >> 8, z = i & 255;
        const int y = r0 + r;
        const float2 Z1 = A[r * N + z];
        const float2 Z2 = A[(RBn + (r >> 1)) * N + z];
        const float psi = Z1.x, dz = Z1.y, dy = (r & 1) ? Z2.y : Z2.x;
        const long long o = base + (long long)y * N + z;
        const int q = y * N + z;
        const float S = a.coef * (a.nb0[q] * (psi - pnp[u]) + a.gy[q] * dy + a.gz[q] * dz);
        const float g = fmaf(a.h, S, pg[u]);
        const float n = fmaf(a.dt, g, pnb[u]);
        __stcg(a.G + o, g);
        __stcg(a.nb + o, n);
        bad |= !(fabsf(n) <= 3.0e38f) || !(fabsf(g) <= 3.0e38f);
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

constexpr size_t SMEM_K1_256 = sizeof(float2) * (256 + 16 * 256 + 16 * 272);
constexpr size_t SMEM_K2_256 = sizeof(float2) * (256 + 2 * 16 * 257 + 16 * 272);
constexpr size_t SMEM_K3_256 = sizeof(float2) * (256 + 24 * 256 + 16 * 272);

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
    r2::k_plasma<<<(unsigned)((c->P + 127) / 128), 128, 0, c->stream>>>(
        c->nb, c->np, c->P, p.n_xi, q, (float)std::cos(D), (float)std::sin(D), (float)std::cos(0.5 * D),
        (float)std::sin(0.5 * D));
    constexpr int NH = N / 2 + 1;
    r2::PushArgs a{c->np, c->nb, c->G, c->nb0, c->gy, c->gz,
                   (float)(-p.species.q / (p.species.m * p.gamma_b)), h, (float)p.dt, (float)p.L_perp, c->err};
    if constexpr (N == 256) {
        r2::k_rowfft256<<<dim3(256 / 32, p.n_xi), 256, SMEM_K1_256, c->stream>>>(c->np, c->S1);
        r2::k_colfft256<<<dim3((129 + 15) / 16, p.n_xi), 256, SMEM_K2_256, c->stream>>>(
            c->S1, c->T1, c->T2, (float)p.L_perp, (float)p.L_perp);
        r2::k_rowinv_push256<<<dim3(256 / 16, p.n_xi), 256, SMEM_K3_256, c->stream>>>(c->T1, c->T2, a);
        c->launches += 4;
        return cudaGetLastError();
    }
    r2::k_rowfft<N, RB><<<dim3(N / RB, p.n_xi), 256, smem_k1<N>(), c->stream>>>(c->np, c->S1);
    r2::k_colfft<N, CB><<<dim3((NH + CB - 1) / CB, p.n_xi), 256, smem_k2<N>(), c->stream>>>(
        c->S1, c->T1, c->T2, (float)p.L_perp, (float)p.L_perp);
    r2::k_rowinv_push<N, RB><<<dim3(N / RB, p.n_xi), 256, smem_k3<N>(), c->stream>>>(c->T1, c->T2, a);
    c->launches += 4;
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
    cudaError_t e = cudaMemcpy(c->nb0, t.data(), sizeof(float) * t.size(), cudaMemcpyHostToDevice);
    if (!e) e = cudaMemset(c->err, 0, sizeof(int) * 4);
    if (!e) e = cudaMemset(c->nb, 0, sizeof(float) * c->cells);
    if (!e) e = cudaMemset(c->G, 0, sizeof(float) * c->cells);
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
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return QS_ERR_CUDA;
    int e = 0;
    if (cudaMemcpy(&e, c->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return QS_ERR_CUDA;
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
