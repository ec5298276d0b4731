/*
 * CPU oracle for the FX-correlator X-engine.  TEST INFRASTRUCTURE ONLY.
 *
 * This file is the plain, slow, obviously correct definition of what the
 * GPU X-engine computes.  It is called only from the test-suite, from the
 * smoke check and from the CPU-baseline leg of the benchmark; no product
 * code path links or executes it.  It shares no code, header, table or
 * constant with the CUDA library: it has its own nibble decoder and its own
 * triangle indexing.
 *
 * What it computes.  The paper's section "Packet capture implementation"
 * fixes the F-engine samples as complex values with a signed 4-bit real and a
 * signed 4-bit imaginary part; its section "Back end" names a linear-algebra
 * module for matrix products, and "Some included blocks" names the unpack and
 * accumulate blocks.  The X-engine is the product of those pieces:
 *
 *   input   x[t][c][i], one byte per complex sample, t-slowest, i-fastest:
 *           high nibble = real part, low nibble = imaginary part, each a
 *           4-bit two's-complement integer in [-8, 7].
 *   output  for every channel c and every input pair i >= j
 *             V_c[i][j] = sum_t x[t][c][i] * conj(x[t][c][j])
 *           i.e. with x = a + i b:
 *             Re V = sum_t (a_i a_j + b_i b_j)
 *             Im V = sum_t (b_i a_j - a_i b_j)
 *           stored as int64 (re, im) pairs, channel-major, packed lower
 *           triangle row-major: index(i, j) = i (i + 1) / 2 + j.
 *
 * Every sum is an exact int64 sum, so the oracle is the exact result; the
 * GPU kernels must reproduce it bit for bit.
 *
 * Parity pins (tests/test_oracle.py): exhaustive decode of all 256 bytes
 * against an encoder-inverted table; all 65536 byte pairs of a 2-input,
 * 1-sample correlation against Python complex-integer products; Hermitian
 * symmetry of the full-square mode; real non-negative autocorrelations;
 * the rank-1 closed form for an identical signal on every input; time and
 * input permutation invariance; gulp splitting; brute force against an
 * independent numpy int64 einsum.
 */
#include <pthread.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Decode one 4-bit two's-complement nibble (0..15) to its signed value.
 * Values 0..7 are themselves; 8..15 stand for -8..-1. */
static int oracle_nibble_value(unsigned nib)
{
    nib &= 0xFu;
    return (nib < 8u) ? (int)nib : (int)nib - 16;
}

/* Unpack one 4+4 sample: real from the high nibble, imaginary from the low. */
void oracle_decode_byte(uint8_t b, int *re, int *im)
{
    *re = oracle_nibble_value((unsigned)b >> 4);
    *im = oracle_nibble_value((unsigned)b);
}

/* Unpack n samples into interleaved signed 8-bit (re, im) pairs: the 4+4 to
 * 8+8 conversion the TBN pipeline performs before its T-engine. */
void oracle_unpack(const uint8_t *packed, size_t n, int8_t *out)
{
    for (size_t k = 0; k < n; ++k) {
        int re, im;
        oracle_decode_byte(packed[k], &re, &im);
        out[2 * k + 0] = (int8_t)re;
        out[2 * k + 1] = (int8_t)im;
    }
}

typedef struct {
    const uint8_t *x;
    int64_t ntime, nchan, ninput;
    int64_t *out;
    int full_square;          /* 0: packed lower triangle; 1: N x N square */
    int64_t chan_begin, chan_end;
} oracle_job;

/* The triple loop over (channel, baseline, time), for a range of channels. */
static void *oracle_correlate_range(void *arg)
{
    const oracle_job *job = (const oracle_job *)arg;
    const int64_t T = job->ntime, C = job->nchan, N = job->ninput;
    const int64_t nbl = job->full_square ? N * N : N * (N + 1) / 2;
    for (int64_t c = job->chan_begin; c < job->chan_end; ++c) {
        int64_t *vc = job->out + 2 * nbl * c;
        for (int64_t i = 0; i < N; ++i) {
            const int64_t jmax = job->full_square ? N - 1 : i;
            for (int64_t j = 0; j <= jmax; ++j) {
                int64_t re = 0, im = 0;
                for (int64_t t = 0; t < T; ++t) {
                    int ai, bi, aj, bj;
                    oracle_decode_byte(job->x[(t * C + c) * N + i], &ai, &bi);
                    oracle_decode_byte(job->x[(t * C + c) * N + j], &aj, &bj);
                    /* x_i * conj(x_j) = (ai + i bi)(aj - i bj) */
                    re += (int64_t)ai * aj + (int64_t)bi * bj;
                    im += (int64_t)bi * aj - (int64_t)ai * bj;
                }
                const int64_t idx = job->full_square ? i * N + j
                                                     : i * (i + 1) / 2 + j;
                vc[2 * idx + 0] = re;
                vc[2 * idx + 1] = im;
            }
        }
    }
    return NULL;
}

/*
 * Correlate one gulp.  x: uint8[ntime][nchan][ninput].  out: int64 pairs,
 * [nchan][ninput (ninput + 1) / 2][2] (full_square = 0) or
 * [nchan][ninput][ninput][2] (full_square = 1, every ordered pair, used only
 * to check Hermitian symmetry).  Channels are split over nthreads POSIX
 * threads; each channel is computed by exactly one thread, so the result
 * does not depend on the thread count.  Returns 0, or -1 on bad arguments.
 */
int oracle_correlate(const uint8_t *x, int64_t ntime, int64_t nchan,
                     int64_t ninput, int64_t *out, int full_square,
                     int nthreads)
{
    if (!x || !out || ntime < 0 || nchan < 0 || ninput < 0) return -1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > nchan) nthreads = nchan > 0 ? (int)nchan : 1;
    oracle_job *jobs = (oracle_job *)calloc((size_t)nthreads, sizeof(oracle_job));
    pthread_t *tids = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !tids) { free(jobs); free(tids); return -1; }
    for (int k = 0; k < nthreads; ++k) {
        jobs[k].x = x; jobs[k].ntime = ntime; jobs[k].nchan = nchan;
        jobs[k].ninput = ninput; jobs[k].out = out;
        jobs[k].full_square = full_square;
        jobs[k].chan_begin = nchan * k / nthreads;
        jobs[k].chan_end = nchan * (k + 1) / nthreads;
    }
    int started = 0;
    for (int k = 1; k < nthreads; ++k) {
        if (pthread_create(&tids[k], NULL, oracle_correlate_range, &jobs[k]) != 0) break;
        started = k;
    }
    oracle_correlate_range(&jobs[0]);
    for (int k = 1; k <= started; ++k) pthread_join(tids[k], NULL);
    /* any range whose thread failed to start is computed here */
    for (int k = started + 1; k < nthreads; ++k) oracle_correlate_range(&jobs[k]);
    free(jobs); free(tids);
    return 0;
}

/*
 * One visibility, computed on its own: channel c, inputs i >= j (or any
 * ordered pair).  Used to check sampled outputs of full-size GPU runs
 * without computing every baseline on the CPU.
 */
void oracle_correlate_one(const uint8_t *x, int64_t ntime, int64_t nchan,
                          int64_t ninput, int64_t c, int64_t i, int64_t j,
                          int64_t *re_out, int64_t *im_out)
{
    int64_t re = 0, im = 0;
    for (int64_t t = 0; t < ntime; ++t) {
        int ai, bi, aj, bj;
        oracle_decode_byte(x[(t * nchan + c) * ninput + i], &ai, &bi);
        oracle_decode_byte(x[(t * nchan + c) * ninput + j], &aj, &bj);
        re += (int64_t)ai * aj + (int64_t)bi * bj;
        im += (int64_t)bi * aj - (int64_t)ai * bj;
    }
    *re_out = re;
    *im_out = im;
}
