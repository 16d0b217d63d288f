// Shared-memory Stockham FFT for power-of-two lengths, executed by a whole CTA.
//
// NB independent sequences of length L lie back to back in shared memory
// (element k of sequence s at logical index s * L + k, see spad below). Each stage of radix R reads the
// R inputs of every butterfly into registers, synchronises, applies the
// twiddles and a radix-R DFT in registers and writes the outputs to their
// auto-sorted positions, then synchronises again; one buffer therefore serves
// every stage. Radix 8 is used while at least 8 points remain per sub-transform,
// then one radix-4 or radix-2 stage.
//
// Stage with span NS (product of the radices before it) and radix R, for the
// butterfly j in [0, L/R) of a sequence, k = j mod NS:
//     v_r = x[j + r L/R] * W_{NS R}^{r k},   r = 0..R-1
//     X = DFT_R(v)
//     y[(j / NS) NS R + k + r NS] = X_r
// (the Stockham auto-sort formulation; the output is in natural order).
//
// Twiddles: a compact table per length L holds, for every stage with span
// NS > 1, the NS values W_{NS R}^k = exp(-2 pi i k / (NS R)), k < NS, built in
// FP64 on the device (sincospi) and cast for FP32 plans; the stages' tables lie
// back to back (spans 8, 64, 512, ... so the table of span NS starts at
// (NS - 8) / 7). A butterfly loads W^k once (consecutive k: a coalesced load)
// and forms W^{2k} .. W^{7k} by complex products of depth at most 3. The
// inverse transform uses the conjugates and is not normalised.
//
// Shared-memory layout: element i of the batch is stored at spad(i), which
// inserts one padding element every 16 (8-byte complex) or 8 (16-byte complex)
// elements so that the strided stores of the early stages fall in distinct
// banks (for a warp, about 1.1x the conflict-free wavefront count instead of
// 2x). Every access to an FFT buffer goes through spad; spad_size(n) is the
// number of elements a buffer holding n logical elements needs.
#pragma once

#include "common.cuh"

template <typename C>
__host__ __device__ __forceinline__ constexpr int spad(int i)
{
    return sizeof(C) == 8 ? i + (i >> 4) : i + (i >> 3);
}

// elements per padding group: spad(i + g m) = spad(i) + m spad(g) for whole groups
template <typename C>
__host__ __device__ __forceinline__ constexpr int spad_group()
{
    return sizeof(C) == 8 ? 16 : 8;
}

template <typename C>
__host__ __device__ __forceinline__ constexpr int spad_size(int n)
{
    return spad<C>(n - 1) + 1;
}

template <typename C, bool INV>
__device__ __forceinline__ C twiddle(const C *__restrict__ tw, int idx)
{
    C w = __ldg(&tw[idx]);
    if (INV) w.y = -w.y;
    return w;
}

// offset of the stage table of span NS (NS = 8, 64, 512, ...) in the compact table
__host__ __device__ constexpr int stage_table_offset(int NS) { return (NS - 8) / 7; }

// entries of the compact table of a length-L transform
__host__ __device__ constexpr int stage_table_size(int L)
{
    int total = 0;
    for (int ns = 1; ns < L;) {
        const int r = L / ns >= 8 ? 8 : L / ns;
        if (ns > 1) total += ns;
        ns *= r;
    }
    return total;
}

// multiply by -i (forward) or +i (inverse)
template <typename C, bool INV>
__device__ __forceinline__ C rot90(C a)
{
    return INV ? cmake<C>(-a.y, a.x) : cmake<C>(a.y, -a.x);
}

template <typename C, bool INV>
__device__ __forceinline__ void dft2(C &a, C &b)
{
    C t = a;
    a = cadd(t, b);
    b = csub(t, b);
}

template <typename C, bool INV>
__device__ __forceinline__ void dft4(C &v0, C &v1, C &v2, C &v3)
{
    C t0 = cadd(v0, v2), t1 = csub(v0, v2);
    C t2 = cadd(v1, v3), t3 = rot90<C, INV>(csub(v1, v3));
    v0 = cadd(t0, t2);
    v2 = csub(t0, t2);
    v1 = cadd(t1, t3);
    v3 = csub(t1, t3);
}

template <typename C, bool INV>
__device__ __forceinline__ void dft8(C *v)
{
    using T = decltype(C::x);
    const T s = (T)0.70710678118654752440;  // 1/sqrt(2)
    C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<C, INV>(e0, e1, e2, e3);
    dft4<C, INV>(o0, o1, o2, o3);
    // o_k *= W8^k, W8 = exp(-+ 2 pi i / 8)
    C w1 = INV ? cmake<C>(s * (o1.x - o1.y), s * (o1.x + o1.y)) : cmake<C>(s * (o1.x + o1.y), s * (o1.y - o1.x));
    C w2 = rot90<C, INV>(o2);
    C w3 = INV ? cmake<C>(-s * (o3.x + o3.y), s * (o3.x - o3.y)) : cmake<C>(s * (o3.y - o3.x), -s * (o3.x + o3.y));
    v[0] = cadd(e0, o0);
    v[4] = csub(e0, o0);
    v[1] = cadd(e1, w1);
    v[5] = csub(e1, w1);
    v[2] = cadd(e2, w2);
    v[6] = csub(e2, w2);
    v[3] = cadd(e3, w3);
    v[7] = csub(e3, w3);
}

// IN_HALF: the first stage takes the inputs at logical positions >= L/2 as
// zero without reading them (zero padding to at least twice the data length).
// OUT_HALF: the last stage writes only the outputs at positions < L/2.
template <typename C, int L, int NB, int THREADS, int NS, int R, bool INV, bool IN_HALF = false, bool OUT_HALF = false>
__device__ __forceinline__ void fft_stage(C *buf, const C *__restrict__ tw)
{
    constexpr int NBF = NB * (L / R);            // butterflies in the stage
    constexpr int PER = (NBF + THREADS - 1) / THREADS;
    C v[PER][R];
    // the R inputs of a butterfly lie L/R apart; when L/R is a whole number of
    // padding groups their padded positions lie a constant distance apart too
    constexpr int S = L / R;
    constexpr bool SPAN_IN = S % spad_group<C>() == 0;
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int b = threadIdx.x + p * THREADS;
        if (NBF % THREADS == 0 || b < NBF) {
            const int seq = b / S, j = b % S;
            const C *src = buf + spad<C>(seq * L + j);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (IN_HALF && NS == 1 && r >= R / 2) v[p][r] = cmake<C>(0, 0);
                else if constexpr (SPAN_IN) v[p][r] = src[r * spad<C>(S)];
                else v[p][r] = buf[spad<C>(seq * L + j + r * S)];
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int b = threadIdx.x + p * THREADS;
        if (NBF % THREADS == 0 || b < NBF) {
            const int seq = b / (L / R), j = b % (L / R);
            const int k = j % NS;
            if constexpr (NS > 1) {
                const C w1 = twiddle<C, INV>(tw, stage_table_offset(NS) + k);
                v[p][1] = cmul(v[p][1], w1);
                if constexpr (R >= 4) {
                    const C w2 = cmul(w1, w1);
                    const C w3 = cmul(w2, w1);
                    v[p][2] = cmul(v[p][2], w2);
                    v[p][3] = cmul(v[p][3], w3);
                    if constexpr (R == 8) {
                        const C w4 = cmul(w2, w2);
                        v[p][4] = cmul(v[p][4], w4);
                        v[p][5] = cmul(v[p][5], cmul(w4, w1));
                        v[p][6] = cmul(v[p][6], cmul(w3, w3));
                        v[p][7] = cmul(v[p][7], cmul(w4, w3));
                    }
                }
            }
            if constexpr (R == 8) dft8<C, INV>(v[p]);
            else if constexpr (R == 4) dft4<C, INV>(v[p][0], v[p][1], v[p][2], v[p][3]);
            else dft2<C, INV>(v[p][0], v[p][1]);
            const int base = seq * L + (j / NS) * NS * R + k;
            constexpr bool SPAN_OUT = NS % spad_group<C>() == 0;
            C *dst = buf + spad<C>(base);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (OUT_HALF && NS * R == L && r >= R / 2) continue;  // position k + r NS >= L/2
                if constexpr (SPAN_OUT) dst[r * spad<C>(NS)] = v[p][r];
                else buf[spad<C>(base + r * NS)] = v[p][r];
            }
        }
    }
    __syncthreads();
}

template <typename C, int L, int NB, int THREADS, int NS, bool INV, bool IN_HALF, bool OUT_HALF>
__device__ __forceinline__ void fft_stages(C *buf, const C *__restrict__ tw)
{
    if constexpr (NS < L) {
        constexpr int REM = L / NS;
        constexpr int R = REM >= 8 ? 8 : REM;
        fft_stage<C, L, NB, THREADS, NS, R, INV, IN_HALF, OUT_HALF>(buf, tw);
        fft_stages<C, L, NB, THREADS, NS * R, INV, IN_HALF, OUT_HALF>(buf, tw);
    }
}

// FFT of NB sequences of length L in shared memory by THREADS threads.
// Must be called by every thread of the CTA (it synchronises). The caller
// synchronises before the call so that the inputs are visible. With IN_HALF
// the inputs at positions >= L/2 are taken as zero (and need not be written);
// with OUT_HALF only the outputs at positions < L/2 are produced.
template <typename C, int L, int NB, int THREADS, bool INV, bool IN_HALF = false, bool OUT_HALF = false>
__device__ __forceinline__ void fft_batch(C *buf, const C *__restrict__ tw)
{
    fft_stages<C, L, NB, THREADS, 1, INV, IN_HALF, OUT_HALF>(buf, tw);
}

// ------------------------------------------------- register-resident form --
//
// The same stages with the data kept in registers between them, for CTAs of
// NSEQ * L / 8 threads (eight elements per thread). Thread t works on sequence
// seq = t / (L/8) and holds, at the start and at the end of a transform, the
// elements of the "pattern P0": v[m] = element jt + m L/8 of its sequence,
// jt = t mod (L/8), m = 0..7. That is the input pattern of a radix-8 first
// stage (butterfly j = jt reads j + r L/8) and the output pattern of the last
// stage (butterfly j writes j + r NS with NS = L/R; a last stage of radix R < 8
// gives thread t the butterflies jt + p L/8, p < 8/R, so that its outputs are
// again P0). Consequences: a transform needs no shared memory before its first
// stage or after its last (loads and stores to global memory go straight to
// and from registers), a forward transform's outputs are the inputs of an
// inverse transform of the same thread with no exchange in between, and
// between two stages one exchange through shared memory (outputs written to
// their auto-sorted positions, a barrier, next inputs read). With NBUF = 2 the
// exchanges alternate between two buffers (one barrier each; `par` carries the
// buffer parity from one transform to the next); with NBUF = 1 a second
// barrier separates each exchange's reads from the next one's writes. Every
// butterfly does the arithmetic of fft_stage (same twiddles, same radix-R
// DFT), so the results are those of fft_batch.
template <typename C, int L, int NSEQ, int THREADS, int NS, int NBUF, bool INV>
__device__ __forceinline__ void rfft_stages(C (&v)[8], C *bufs, int &par, const C *__restrict__ tw)
{
    static_assert(THREADS == NSEQ * L / 8, "eight elements per thread");
    if constexpr (NS < L) {
        constexpr int REM = L / NS;
        constexpr int R = REM >= 8 ? 8 : REM;
        constexpr int PER = 8 / R;
        constexpr int S = L / R;
        constexpr int BUF = spad_size<C>(NSEQ * L);
        const int seq = threadIdx.x / (L / 8), jt = threadIdx.x % (L / 8);
        if constexpr (NS > 1) {
            // gather this stage's inputs from the previous stage's outputs
            const C *in = bufs + (NBUF == 2 ? (par ^ 1) * BUF : 0);
#pragma unroll
            for (int p = 0; p < PER; ++p)
#pragma unroll
                for (int r = 0; r < R; ++r) v[p * R + r] = in[spad<C>(seq * L + jt + p * (L / 8) + r * S)];
            if constexpr (NBUF == 1) __syncthreads();
        }
#pragma unroll
        for (int p = 0; p < PER; ++p) {
            C *u = v + p * R;
            const int j = jt + p * (L / 8);
            const int k = j % NS;
            if constexpr (NS > 1) {
                const C w1 = twiddle<C, INV>(tw, stage_table_offset(NS) + k);
                u[1] = cmul(u[1], w1);
                if constexpr (R >= 4) {
                    const C w2 = cmul(w1, w1);
                    const C w3 = cmul(w2, w1);
                    u[2] = cmul(u[2], w2);
                    u[3] = cmul(u[3], w3);
                    if constexpr (R == 8) {
                        const C w4 = cmul(w2, w2);
                        u[4] = cmul(u[4], w4);
                        u[5] = cmul(u[5], cmul(w4, w1));
                        u[6] = cmul(u[6], cmul(w3, w3));
                        u[7] = cmul(u[7], cmul(w4, w3));
                    }
                }
            }
            if constexpr (R == 8) dft8<C, INV>(u);
            else if constexpr (R == 4) dft4<C, INV>(u[0], u[1], u[2], u[3]);
            else dft2<C, INV>(u[0], u[1]);
        }
        if constexpr (NS * R == L) {
            // last stage: butterfly jt + p L/8, output r at jt + (p + r PER) L/8
            C o[8];
#pragma unroll
            for (int p = 0; p < PER; ++p)
#pragma unroll
                for (int r = 0; r < R; ++r) o[p + r * PER] = v[p * R + r];
#pragma unroll
            for (int m = 0; m < 8; ++m) v[m] = o[m];
        } else {
            C *out = bufs + (NBUF == 2 ? par * BUF : 0);
#pragma unroll
            for (int p = 0; p < PER; ++p) {
                const int j = jt + p * (L / 8);
                const int base = seq * L + (j / NS) * NS * R + j % NS;
#pragma unroll
                for (int r = 0; r < R; ++r) out[spad<C>(base + r * NS)] = v[p * R + r];
            }
            __syncthreads();
            if constexpr (NBUF == 2) par ^= 1;
            rfft_stages<C, L, NSEQ, THREADS, NS * R, NBUF, INV>(v, bufs, par, tw);
        }
    }
}

// Transform of the P0-held data of every thread's sequence (see above). Every
// thread of the CTA calls it. bufs: NBUF buffers of spad_size(NSEQ L) elements.
// With NBUF = 1 the caller must make sure that no thread still reads the
// buffer from an earlier use when this call starts writing it.
template <typename C, int L, int NSEQ, int THREADS, int NBUF, bool INV>
__device__ __forceinline__ void fft_regs(C (&v)[8], C *bufs, int &par, const C *__restrict__ tw)
{
    rfft_stages<C, L, NSEQ, THREADS, 1, NBUF, INV>(v, bufs, par, tw);
}
