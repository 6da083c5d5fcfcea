/*
 * CPU oracle for permuted FHT-FSCL decoding of Reed-Muller codes
 * (Doan, Hashemi, Gross, "Successive-Cancellation Decoding of Reed-Muller Codes with Fast
 * Hadamard Transform", arXiv 2108.12550).
 *
 * TEST INFRASTRUCTURE ONLY. This library is the reference the GPU decoder is checked
 * against. Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
 * load it; the decoder product never does. It shares no code with the GPU path.
 *
 * What it computes, and where the paper defines it:
 *   - min-sum f and g, Section II-B;
 *   - FHTL / FHT decoding of RM(1,s) nodes with the short path metric, Algorithms 3-4 and
 *     Eqs. (7)-(8);
 *   - SPCL decoding of RM(s-1,s) nodes, Eqs. (2)-(6);
 *   - the permuted recursion p-FHT-FSCL, Algorithm 2, and the M parallel decoders with
 *     the smallest-metric selection, Algorithm 5;
 *   - the Aut-SSC-P baseline the paper compares against (Section III-B, Table 5): SSC
 *     decoding of P permuted copies with repetition and SPC nodes, most likely candidate.
 * Readings where the paper is silent or inconsistent (tie rules, the 2L loop bound of
 * Algorithm 2, tau of the SPC node, the codeword convention of the FHT) are stated at the
 * functions that use them. Two arithmetic modes: FP64 (suffix f64) and int64 (suffix i64)
 * for quantised LLRs.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define MAXM 10
#define MAXN (1 << MAXM)
#define PERM_REC 11 /* [c_0 .. c_9, b]: c_t = A e_t, record maps i -> b ^ A v(i) */

static int ga_apply(const uint16_t *rec, int s, int i) {
    int v = rec[MAXM];
    for (int t = 0; t < s; t++)
        if ((i >> t) & 1) v ^= rec[t];
    return v;
}

static int n_perm_levels(int m, int r) { return (1 < r && r < m - 1) ? r - 1 : 0; }
static int perms_per_decoder(int m, int r, int L) { return L + n_perm_levels(m, r) * 2 * L; }

/* u = x G^{(x)m} over GF(2) (G^{(x)m} is its own inverse): u_i = XOR of x_j over j containing i. */
static void polar_transform(uint8_t *v, int m) {
    int n = 1 << m;
    for (int h = 1; h < n; h <<= 1)
        for (int i = 0; i < n; i += 2 * h)
            for (int j = i; j < i + h; j++) v[j] ^= v[j + h];
}

/* Writes the information bits (I ascending); returns 0 if x is a codeword of RM(r,m). */
static int extract_info(const uint8_t *cw, int m, int r, uint8_t *info) {
    int n = 1 << m, q = 0, ok = 1;
    uint8_t u[MAXN];
    memcpy(u, cw, n);
    polar_transform(u, m);
    for (int i = 0; i < n; i++) {
        if (__builtin_popcount((unsigned)i) >= m - r) info[q++] = u[i];
        else if (u[i]) ok = 0;
    }
    return ok ? 0 : -1;
}

#define VAL double
#define SFX f64
#define IS_INT 0
#include "pfht_core.inc"
#undef VAL
#undef SFX
#undef IS_INT

#define VAL int64_t
#define SFX i64
#define IS_INT 1
#include "pfht_core.inc"
#undef VAL
#undef SFX
#undef IS_INT

/* ------------------------------------------------------------------ batch drivers --- */

typedef struct {
    int kind; /* 0 f64 decode, 1 i64 decode, 2 f64 aut-ssc, 3 i64 aut-ssc */
    int m, r, P, L;
    int no_perm; /* FHT-FSCL (no permutations) */
    const uint16_t *perms;
    const void *llr;
    int64_t f0, f1;
    uint8_t *cw_out, *info_out;
    void *pm_out;
    double *margin_out;
    int64_t *ops_out;
    int32_t *best_out;
    int bad; /* frames whose output is not a codeword (must stay 0) */
    int64_t *paper_out; /* the paper's complexity count C per frame, or NULL */
} job_t;

static void *run_job(void *arg) {
    job_t *j = arg;
    int N = 1 << j->m;
    int K = 0;
    for (int i = 0; i < N; i++) K += __builtin_popcount((unsigned)i) >= j->m - j->r;
    void *ba = NULL, *bb = NULL;
    if (j->kind == 0) { ba = calloc(j->L, sizeof(path_t_f64)); bb = calloc(j->L, sizeof(path_t_f64)); }
    if (j->kind == 1) { ba = calloc(j->L, sizeof(path_t_i64)); bb = calloc(j->L, sizeof(path_t_i64)); }
    uint8_t cw[MAXN], info[MAXN];
    for (int64_t f = j->f0; f < j->f1; f++) {
        int best = -1;
        if (j->kind == 0) {
            const double *y = (const double *)j->llr + f * N;
            best = decode_frame_f64(j->m, j->r, j->P, j->L, j->no_perm, j->perms, y, ba, bb, cw,
                                    (double *)j->pm_out + f, j->margin_out ? j->margin_out + f : NULL,
                                    j->ops_out ? j->ops_out + f : NULL, j->paper_out ? j->paper_out + f : NULL);
        } else if (j->kind == 1) {
            const int64_t *y = (const int64_t *)j->llr + f * N;
            best = decode_frame_i64(j->m, j->r, j->P, j->L, j->no_perm, j->perms, y, ba, bb, cw,
                                    (int64_t *)j->pm_out + f, j->margin_out ? j->margin_out + f : NULL,
                                    j->ops_out ? j->ops_out + f : NULL, j->paper_out ? j->paper_out + f : NULL);
        } else if (j->kind == 2) {
            best = aut_ssc_frame_f64(j->m, j->r, j->P, j->perms, (const double *)j->llr + f * N, cw,
                                     (double *)j->pm_out + f);
        } else {
            best = aut_ssc_frame_i64(j->m, j->r, j->P, j->perms, (const int64_t *)j->llr + f * N, cw,
                                     (int64_t *)j->pm_out + f);
        }
        if (extract_info(cw, j->m, j->r, info) != 0) j->bad++;
        if (j->cw_out) memcpy(j->cw_out + f * N, cw, N);
        if (j->info_out) memcpy(j->info_out + f * K, info, K);
        if (j->best_out) j->best_out[f] = best;
    }
    free(ba); free(bb);
    return NULL;
}

static int run_batch(job_t proto, int64_t n_frames, int n_threads) {
    if (proto.m < 2 || proto.m > MAXM || proto.L < 1 || proto.L > 32 || proto.P < 1) return -1;
    if (proto.kind <= 1 && !(1 <= proto.r && proto.r <= proto.m - 1)) return -1;
    if (proto.kind >= 2 && !(0 <= proto.r && proto.r <= proto.m)) return -1;
    if (n_threads <= 0) n_threads = (int)sysconf(_SC_NPROCESSORS_ONLN);
    if (n_threads > n_frames) n_threads = n_frames > 0 ? (int)n_frames : 1;
    pthread_t th[256];
    job_t jobs[256];
    if (n_threads > 256) n_threads = 256;
    for (int t = 0; t < n_threads; t++) {
        jobs[t] = proto;
        jobs[t].f0 = n_frames * t / n_threads;
        jobs[t].f1 = n_frames * (t + 1) / n_threads;
        pthread_create(&th[t], NULL, run_job, &jobs[t]);
    }
    int bad = 0;
    for (int t = 0; t < n_threads; t++) { pthread_join(th[t], NULL); bad += jobs[t].bad; }
    return bad ? -2 : 0;
}

/* p-FHT-FSCL-L-P decoding of n_frames FP64 LLR frames (row-major [n_frames][2^m]).
 * perms: (P, L + (r-1)*2L, 11) uint16 records. Outputs (each may be NULL except pm_out):
 * cw_out [F][N] codeword bits, info_out [F][K] information bits, pm_out [F] winning path
 * metric, margin_out [F] smallest relative gap at any selection boundary, ops_out [F]
 * algorithmic operation count, best_out [F] winning decoder. Returns 0, -1 on bad
 * arguments, -2 if some output was not a codeword. */
int rmo_decode_f64(int m, int r, int P, int L, const uint16_t *perms, const double *llr,
                   int64_t n_frames, int n_threads, uint8_t *cw_out, uint8_t *info_out,
                   double *pm_out, double *margin_out, int64_t *ops_out, int32_t *best_out) {
    job_t j = {0, m, r, P, L, 0, perms, llr, 0, 0, cw_out, info_out, pm_out, margin_out, ops_out, best_out, 0};
    return run_batch(j, n_frames, n_threads);
}

/* FHT-FSCL-L: the same recursion without permutations, starting from one live path (the
 * decoder the paper's p-FHT-FSCL improves on, its Fig. 4 dashed curves); P = 1. integer
 * selects the int64 mode (llr then points to int64 values, pm_out to int64). */
int rmo_decode_fhtfscl(int m, int r, int L, int integer, const void *llr, int64_t n_frames, int n_threads,
                       uint8_t *cw_out, uint8_t *info_out, void *pm_out, double *margin_out) {
    job_t j = {integer ? 1 : 0, m, r, 1, L, 1, NULL, llr, 0, 0, cw_out, info_out, pm_out, margin_out, NULL, NULL, 0};
    return run_batch(j, n_frames, n_threads);
}

/* Both operation counts of p-FHT-FSCL-L-P (no_perm = 0) or FHT-FSCL-L (no_perm = 1, P = 1,
 * perms unused) on FP64 frames: ops_out [F] this build's count (the roofline numerator),
 * paper_out [F] the paper's complexity C (Section III-C, Tables 1-2; see tally in
 * pfht_core.inc). Either output may be NULL. */
int rmo_op_counts(int m, int r, int P, int L, int no_perm, const uint16_t *perms, const double *llr,
                  int64_t n_frames, int n_threads, int64_t *ops_out, int64_t *paper_out) {
    if (no_perm && P != 1) return -1;
    job_t j = {0, m, r, P, L, no_perm ? 1 : 0, perms, llr, 0, 0, NULL, NULL, NULL, NULL, ops_out, NULL, 0, paper_out};
    double *pm = malloc(sizeof(double) * (n_frames > 0 ? n_frames : 1));
    j.pm_out = pm;
    int rc = run_batch(j, n_frames, n_threads);
    free(pm);
    return rc;
}

/* The same decoder in exact int64 arithmetic on integer LLRs (the quantised-LLR mode). */
int rmo_decode_i64(int m, int r, int P, int L, const uint16_t *perms, const int64_t *llr,
                   int64_t n_frames, int n_threads, uint8_t *cw_out, uint8_t *info_out,
                   int64_t *pm_out, double *margin_out, int64_t *ops_out, int32_t *best_out) {
    job_t j = {1, m, r, P, L, 0, perms, llr, 0, 0, cw_out, info_out, pm_out, margin_out, ops_out, best_out, 0};
    return run_batch(j, n_frames, n_threads);
}

/* Aut-SSC-P: perms is (Pssc, 11) GA(m) records; pm_out receives the correlation
 * discrepancy of the chosen codeword. */
int rmo_aut_ssc_f64(int m, int r, int Pssc, const uint16_t *perms, const double *llr,
                    int64_t n_frames, int n_threads, uint8_t *cw_out, uint8_t *info_out,
                    double *disc_out, int32_t *best_out) {
    job_t j = {2, m, r, Pssc, 1, 0, perms, llr, 0, 0, cw_out, info_out, disc_out, NULL, NULL, best_out, 0};
    return run_batch(j, n_frames, n_threads);
}

int rmo_aut_ssc_i64(int m, int r, int Pssc, const uint16_t *perms, const int64_t *llr,
                    int64_t n_frames, int n_threads, uint8_t *cw_out, uint8_t *info_out,
                    int64_t *disc_out, int32_t *best_out) {
    job_t j = {3, m, r, Pssc, 1, 0, perms, llr, 0, 0, cw_out, info_out, disc_out, NULL, NULL, best_out, 0};
    return run_batch(j, n_frames, n_threads);
}

/* ------------------------------------------------------- single-node entry points --- */
/* One FHTL or SPCL node on L given paths (LLRs alpha [L][2^s], metrics pm [L]): returns
 * the L surviving paths as parent index, node codeword bits [L][2^s] and metric. */
static int node_entry_f64(int kind, int s, int L, const double *alpha, const double *pm,
                          int32_t *parent, uint8_t *x, double *pm_out) {
    if (s < 1 || s > MAXM || L < 1 || L > 32) return -1;
    int N = 1 << s;
    path_t_f64 *a = calloc(L, sizeof(path_t_f64)), *b = calloc(L, sizeof(path_t_f64));
    dec_t_f64 d;
    memset(&d, 0, sizeof d);
    d.L = L; d.cur = a; d.nxt = b; d.scale = 1.0; d.margin = INFINITY;
    for (int l = 0; l < L; l++) {
        a[l].pm = pm[l];
        a[l].init = l; /* reused as the parent tag */
        memcpy(a[l].alpha + N, alpha + (size_t)l * N, sizeof(double) * N);
    }
    if (kind == 0) fhtl_f64(&d, s, 0); else spcl_f64(&d, s, 0);
    for (int l = 0; l < L; l++) {
        parent[l] = d.cur[l].init;
        memcpy(x + (size_t)l * N, d.cur[l].x, N);
        pm_out[l] = d.cur[l].pm;
    }
    free(a); free(b);
    return 0;
}

int rmo_fhtl_f64(int s, int L, const double *alpha, const double *pm, int32_t *parent, uint8_t *x, double *pm_out) {
    return node_entry_f64(0, s, L, alpha, pm, parent, x, pm_out);
}
int rmo_spcl_f64(int s, int L, const double *alpha, const double *pm, int32_t *parent, uint8_t *x, double *pm_out) {
    return node_entry_f64(1, s, L, alpha, pm, parent, x, pm_out);
}
