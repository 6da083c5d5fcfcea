// p-FHT-FSCL-L-M for the short codes RM(2, m), 4 <= m <= 8, and RM(3, m), 5 <= m <= 7, with
// one thread per list path (two threads per path for m = 8).
//
// Method: Doan, Hashemi, Gross, arXiv 2108.12550 — Algorithm 2 (the permuted nodes: the root,
// and for RM(3, m) also its left child RM(2, m-1); 2L candidate permutations each, ranked by the
// reliability metric LM), Algorithms 3-4 with Eq. (8) (FHTL nodes RM(1, s)), Eqs. (2)-(6) (the
// SPCL nodes RM(2, 3) and RM(3, 4)) and Algorithm 5 (the best of P decoders).
//
// Execution model. The L paths of one decoder are G L consecutive lanes of a warp (G = 1 lane
// per path, or G = 2 for m = 8: lane g of a path holds its positions i = G e + g); a lane keeps
// its share of the path's LLRs of every pending tree level, the Walsh-Hadamard spectra and the
// path's decided bits in registers (at most 64 + 32 floats), so the tree's f/g steps and
// butterflies run without shared memory (for G = 2 one butterfly stage of each node pairs the
// path's two lanes) and every lane does useful work. Lists interact only at the leaves: the
// survivors are chosen by shuffles among the decoder's lanes, and a new path copies its
// parent's pending LLRs with one shuffle per value. The decoders of a frame occupy a group of
// FW consecutive lanes (FW = G L x decoders per batch, a power of two); a warp decodes 32 / FW
// frames at once and runs the P decoders of each frame in batches of FW / (G L). A CTA of W
// warps takes 32 / FW frames at a time, staged once in its shared memory: warp w runs batches
// w, w + W, ..., and the warps' best decoders meet in shared memory, so that a frame waits for
// ceil(batches / W) batches rather than for all of them.
//
// Results: integer-valued inputs decode bit-exactly as the warp-per-decoder kernel and the
// integer oracle do (every operation is exact there). Sums (the metric LM, sum |alpha| of an
// FHTL node) and butterflies take the warp-per-decoder kernel's association order. A path
// offers its FHTL candidates in the order (|c_k| descending, k ascending); the survivors of a
// leaf are the L smallest by (PM', path, k), PM' = PM + (sum|alpha| - |c_k|) / 2 in FP32.
#pragma once

#include <cstdint>

#include <cuda_fp16.h>

#include "pfht_kernel.cuh"

namespace rmdec_dev {

// Lanes per path: two for m = 8 (the largest leaf's 128 values), else one.
__host__ __device__ constexpr int ppt_lanes_per_path(int m) { return m >= 8 ? 2 : 1; }
// Lanes per frame group: the decoders of one batch (G L lanes each); at least N / 32 lanes, so
// that a warp stages at most 32 N / FW <= 1024 LLRs (4 KB, plus the padding of ppt_frame_stride).
__host__ __device__ constexpr int ppt_pow2_ceil(int x) { return x <= 1 ? 1 : 2 * ppt_pow2_ceil((x + 1) / 2); }
__host__ __device__ inline int ppt_frame_lanes(int m, int L, int P) {
    const int n32 = m >= 5 ? (1 << m) / 32 : 1;
    int fw = ppt_pow2_ceil(P * L * ppt_lanes_per_path(m));
    if (fw > 32) fw = 32;
    if (fw < n32) fw = n32;
    return fw;
}

// Floats between the starts of consecutive staged frames of a warp: N, padded when several
// frames share the warp so that their starts fall on distinct banks, 32 / FPW banks apart (at
// least 4, which keeps every frame 16-byte aligned for the vector loads).
__host__ __device__ inline int ppt_frame_stride(int m, int fpw) {
    const int n = 1 << m;
    if (fpw <= 1) return n;
    const int spacing = 32 / fpw > 4 ? 32 / fpw : 4;
    return n + (((spacing - n) % 32) + 32) % 32;
}
// trailing zeros of 0 < n < 128 (folds to a constant for constant n, unlike a recursion)
__host__ __device__ constexpr int ctz7(int n) {
    return (n & 1) ? 0 : (n & 2) ? 1 : (n & 4) ? 2 : (n & 8) ? 3 : (n & 16) ? 4 : (n & 32) ? 5 : 6;
}

// Batcher's odd-even merge sort network on NS = 2^k inputs (Knuth's formulation), as a
// compile-time list of comparators (19 for NS = 8, 63 for NS = 16), so that the sorting code
// unrolls into straight-line compare-exchanges on registers.
template <int NS>
struct OddEvenMergeNet {
    static constexpr int kMax = 64;
    int n = 0;
    int lo[kMax] = {};
    int hi[kMax] = {};
    constexpr OddEvenMergeNet() {
        for (int pp = 1; pp < NS; pp <<= 1)
            for (int k = pp; k >= 1; k >>= 1)
                for (int j = k % pp; j + k < NS; j += 2 * k)
                    for (int i = 0; i < k; i++)
                        if (i + j + k < NS && (i + j) / (2 * pp) == (i + j + k) / (2 * pp)) {
                            lo[n] = i + j;
                            hi[n] = i + j + k;
                            n++;
                        }
    }
};

// Word `idx` (< NW <= 8) of a register array, by a multiplexer on the index bits (an equality
// chain would be turned into a local-memory array by the compiler).
template <int NW>
__device__ __forceinline__ uint32_t pick_word(const uint32_t (&x)[NW], int idx) {
    if constexpr (NW == 1) {
        return x[0];
    } else if constexpr (NW == 2) {
        return (idx & 1) ? x[1] : x[0];
    } else if constexpr (NW == 4) {
        const uint32_t lo = (idx & 1) ? x[1] : x[0], hi = (idx & 1) ? x[3] : x[2];
        return (idx & 2) ? hi : lo;
    } else {
        static_assert(NW == 8, "one to eight words");
        const uint32_t a = (idx & 1) ? x[1] : x[0], b = (idx & 1) ? x[3] : x[2];
        const uint32_t c = (idx & 1) ? x[5] : x[4], d = (idx & 1) ? x[7] : x[6];
        const uint32_t lo = (idx & 2) ? b : a, hi = (idx & 2) ? d : c;
        return (idx & 4) ? hi : lo;
    }
}

template <int M, int R, int L>
struct Ppt {
    static constexpr int G = ppt_lanes_per_path(M);  // lanes per path
    static constexpr int DL = G * L;                  // lanes per decoder
    static constexpr int N = 1 << M;
    static constexpr int H = N / 2;
    static constexpr int NW = (N + 31) / 32;
    static constexpr int NREC = 2 * L * (R - 1);  // candidate maps per decoder (R - 1 permuted levels)
    // Shared-memory columns (value e of lane t at word 32 e + t): RM(2, m) keeps the LLRs of
    // level m-1 there (m >= 6) while the leaf RM(1, m-2) is decoded, instead of in registers,
    // so that the register peak, and with it the resident warps, follows the largest leaf alone.
    // RM(3, m) keeps there the permuted node's LLRs (the candidates gather from them) and the
    // pending LLRs of its RM(3, s) nodes of levels m-1 and m-2 while their left subtrees run.
    static constexpr bool PEND_SMEM = R == 3 || M >= 6;
    static constexpr int COL1 = (R == 3 && M - 2 >= 5) ? (1 << (M - 2)) : 0;  // level m-2 column
    static constexpr int PEND_FLOATS = PEND_SMEM ? (H / G + COL1) * 32 : 0;   // per warp
    static_assert(M >= 4 && M <= 8, "short codes");
    static_assert(R == 2 || (R == 3 && M >= 5 && M <= 7 && G == 1), "RM(2, m); RM(3, m) for m <= 7");
    static_assert(L == 1 || L == 2 || L == 4 || L == 8, "list size");
    static_assert(DL <= 32, "a decoder within a warp");

    struct Ctx {
        const float* y;         // the frame's LLRs (shared memory)
        const uint16_t* rec;    // the decoder's maps: 2L composed root records, then (R = 3) the
                                // 2L records of the permuted node RM(2, m-1) (shared memory)
        const uint16_t* rinv;   // their inverse maps, in the same order (shared memory)
        uint8_t* sel;           // the warp's 32-byte selection scratch
        float* pend;            // the warp's level-(m-1) LLRs: value e of lane t at [32 e + t]
        int dbase;              // lane of the decoder's path 0
        int l;                  // this lane's path
        int g;                  // this lane within its path (positions G e + g)
        bool single;            // paths 1..L-1 start inactive (metric +inf)
        bool int8;              // INT8 LLR codes (every tree value an integer, see fht_leaf)
    };
    struct Path {
        float pm;
        int rootc;         // root candidate (composed permutation) the path descends from
        int selc;          // R = 3: the candidate chosen at the permuted node RM(2, m-1)
        int own[2];        // R = 3: lanes whose columns hold the ancestors' pending LLRs
        uint32_t x[NW];    // decided bits of the permuted word, span layout of the tree
    };

    // bit i of the decided word
    __device__ __forceinline__ static unsigned bit(const Path& p, int i) { return (p.x[i >> 5] >> (i & 31)) & 1u; }
    // bit G e + g, for a compile-time G e (the word is known; the lane's g shifts)
    __device__ __forceinline__ static unsigned bitg(const Path& p, int ge, int g) {
        return (p.x[ge >> 5] >> ((ge & 31) + g)) & 1u;
    }
    // the lane of path `path` holding this lane's positions
    __device__ __forceinline__ static int lane_of(const Ctx& c, int path) { return c.dbase + G * path + c.g; }

    // Writes the NB bits `v` at span offset OFF (NB <= 32 and OFF a multiple of NB, or NB a
    // multiple of 32 with v holding word `wd`).
    template <int OFF, int NB>
    __device__ __forceinline__ static void put_bits(Path& p, unsigned v) {
        static_assert(NB <= 32 && OFF % NB == 0, "small span");
        constexpr unsigned mask = (NB == 32 ? 0xffffffffu : ((1u << NB) - 1u)) << (OFF % 32);
        p.x[OFF / 32] = (p.x[OFF / 32] & ~mask) | ((v << (OFF % 32)) & mask);
    }

    // x_v = (x_gamma ^ x_lambda, x_gamma) on the span [OFF, OFF + 2 HS) (Algorithm 2)
    template <int OFF, int HS>
    __device__ __forceinline__ static void combine(Path& p) {
        if constexpr (HS >= 32) {
#pragma unroll
            for (int w = 0; w < HS / 32; w++) p.x[OFF / 32 + w] ^= p.x[(OFF + HS) / 32 + w];
        } else {
            constexpr unsigned mh = (1u << HS) - 1u;
            p.x[OFF / 32] ^= ((p.x[OFF / 32] >> ((OFF % 32) + HS)) & mh) << (OFF % 32);
        }
    }

    // New path (this lane) descends from path `par`: its root candidate, the pending LLRs
    // `pend` (PC values) and the decided bits left of span offset OFF.
    template <int OFF, int PC, int PA>
    __device__ __forceinline__ static void list_step(const Ctx& c, Path& p, int par, float (&pend)[PA]) {
        const int src = lane_of(c, par);
        p.rootc = __shfl_sync(kFull, p.rootc, src);
        if constexpr (R == 3) {
            p.selc = __shfl_sync(kFull, p.selc, src);
            p.own[0] = __shfl_sync(kFull, p.own[0], src);
            p.own[1] = __shfl_sync(kFull, p.own[1], src);
        }
#pragma unroll
        for (int i = 0; i < PC; i++) pend[i] = __shfl_sync(kFull, pend[i], src);
#pragma unroll
        for (int w = 0; w < (OFF + 31) / 32; w++) p.x[w] = __shfl_sync(kFull, p.x[w], src);
    }

    // --------------------------------------------------------------- FHTL leaf ---
    // RM(1, S) node at span offset OFF (Algorithms 3-4, Eq. (8)): spectrum c = H alpha, path
    // candidates (k, sign of c_k) with PM' = PM + (sum|alpha| - |c_k|) / 2; the L best over the
    // decoder's paths by (PM', path, k) survive. pend: the PC pending LLRs a new path copies.
    template <int S, int OFF, int PC, int PA>
    __device__ __forceinline__ static int fht_leaf(const Ctx& c, Path& p, float (&v)[(1 << S) / G], float (&pend)[PA]) {
        constexpr int NS = 1 << S;
        constexpr int VS = NS / G;      // this lane's values: positions G e + g
        constexpr int T = cmin(L, VS);  // candidates a lane offers (all of a path's L best)
        // the warp-per-decoder kernel's lanes per path (GO) and values per lane (EO): sums and
        // butterflies below associate as its lane and register steps do; its lane go holds
        // positions go + GO eo, here in the lane g = go mod G, at e = go / G + (GO / G) eo
        constexpr int GO = cmin(32 / L, NS);
        constexpr int EO = NS / GO;
        constexpr int HO = GO / G;  // its lanes whose positions this lane holds
        static_assert(GO % G == 0, "whole lanes of that kernel per lane");
        float A;
        {
            float tg[HO];
#pragma unroll
            for (int ho = 0; ho < HO; ho++) {
                float t[EO];
#pragma unroll
                for (int e = 0; e < EO; e++) t[e] = fabsf(v[ho + HO * e]);
#pragma unroll
                for (int h = EO / 2; h >= 1; h >>= 1)
#pragma unroll
                    for (int e = 0; e < h; e++) t[e] += t[e + h];
                tg[ho] = t[0];
            }
            if constexpr (G == 2) {
#pragma unroll
                for (int ho = 0; ho < HO; ho++) tg[ho] += __shfl_xor_sync(kFull, tg[ho], 1);
            }
#pragma unroll
            for (int d = 1; d < HO; d <<= 1)
#pragma unroll
                for (int ho = 0; ho < HO; ho += 2 * d) tg[ho] += tg[ho + d];
            A = tg[0];
        }
        // butterflies (u, w) -> (u + w, u - w): index bits of eo, then of go
#pragma unroll
        for (int h = 1; h < EO; h <<= 1)
#pragma unroll
            for (int e = 0; e < EO; e++)
                if (!(e & h))
#pragma unroll
                    for (int ho = 0; ho < HO; ho++) {
                        const float a = v[ho + HO * e], b = v[ho + HO * (e + h)];
                        v[ho + HO * e] = a + b;
                        v[ho + HO * (e + h)] = a - b;
                    }
#pragma unroll
        for (int d = 1; d < GO; d <<= 1) {
            if (d < G) {
                // positions i and i ^ 1 sit in the path's two lanes: lower u + w, upper u - w
                const float sg = c.g ? -1.f : 1.f;
#pragma unroll
                for (int e = 0; e < VS; e++) v[e] = fmaf(sg, v[e], __shfl_xor_sync(kFull, v[e], 1));
            } else {
                const int dl = d / G;
#pragma unroll
                for (int e = 0; e < VS; e++)
                    if (((e % HO) & dl) == 0) {
                        const float a = v[e], b = v[e + dl];
                        v[e] = a + b;
                        v[e + dl] = a - b;
                    }
            }
        }
        // this lane's T best candidates by (|c_k| descending, k ascending): a scan in k order
        // (k = G e + g) inserts before the first entry of strictly smaller |c|; entries hold |c|
        // (sentinel -1) and 2k + [c_k < 0]
        float tv[T];
        unsigned tk[T];
        if (M >= 6 && c.int8) {
            // (codes of length 32 and less keep the one list form: this one measured 1.5%
            // slower there, its extra code outweighing the leaves' few values)
            // INT8 codes: every |c_k| is an integer of at most 2^m x 128 <= 2^15 (each tree
            // level at most doubles an LLR, a length-2^s transform at depth m - s multiplies it
            // by at most 2^s), so its FP32 pattern has at least 8 zero low bits. They take
            // (VS - 1 - e, [c_k < 0]), which turns (|c| descending, e ascending) into the
            // descending order of one integer: the list update is a max/min network
            constexpr int EB = cilog2(VS);
            static_assert(M <= 8 && 1 + EB <= 8, "index and sign fit the zero low bits");
            constexpr unsigned LOW = (2u << EB) - 1u;
            unsigned pk[T];
#pragma unroll
            for (int j = 0; j < T; j++) pk[j] = 0u;  // below every key (VS >= T keys follow)
#pragma unroll
            for (int e = 0; e < VS; e++) {
                const unsigned b = __float_as_uint(v[e]);
                const unsigned x = (b & 0x7fffffffu) | ((unsigned)(VS - 1 - e) << 1) | (b > 0x80000000u ? 1u : 0u);
                unsigned np[T];
                np[0] = umax(pk[0], x);
#pragma unroll
                for (int j = 1; j < T; j++) np[j] = umax(pk[j], umin(pk[j - 1], x));
#pragma unroll
                for (int j = 0; j < T; j++) pk[j] = np[j];
            }
#pragma unroll
            for (int j = 0; j < T; j++) {
                tv[j] = __uint_as_float(pk[j] & ~LOW);
                const unsigned e = (unsigned)(VS - 1) - ((pk[j] >> 1) & (unsigned)(VS - 1));
                tk[j] = 2u * (G * e + (unsigned)c.g) + (pk[j] & 1u);
            }
        } else {
#pragma unroll
            for (int j = 0; j < T; j++) {
                tv[j] = -1.f;
                tk[j] = 2u * (G * j + c.g);
            }
#pragma unroll
            for (int e = 0; e < VS; e++) {
                const float x = fabsf(v[e]);
                const unsigned xk = 2u * (G * e + c.g) + (v[e] < 0.f ? 1u : 0u);
                // the new list from the old one: entry j keeps, takes x, or takes entry j - 1
                bool gt[T];
#pragma unroll
                for (int j = 0; j < T; j++) gt[j] = x > tv[j];
                float ntv[T];
                unsigned ntk[T];
                ntv[0] = gt[0] ? x : tv[0];
                ntk[0] = gt[0] ? xk : tk[0];
#pragma unroll
                for (int j = 1; j < T; j++) {
                    ntv[j] = gt[j - 1] ? tv[j - 1] : (gt[j] ? x : tv[j]);
                    ntk[j] = gt[j - 1] ? tk[j - 1] : (gt[j] ? xk : tk[j]);
                }
#pragma unroll
                for (int j = 0; j < T; j++) {
                    tv[j] = ntv[j];
                    tk[j] = ntk[j];
                }
            }
        }
        // keys (PM', path 2^(S+1) + 2k + sign) of the lane's list, in ascending order
        unsigned key[T], cid[T];
#pragma unroll
        for (int j = 0; j < T; j++) {
            key[j] = ordered_bits(p.pm + 0.5f * (A - tv[j]));
            cid[j] = ((unsigned)c.l << (S + 1)) | tk[j];
        }
        unsigned mkey = key[0], mcid = cid[0];
        if constexpr (DL > 1) {
            // L rounds of the decoder-wide minimum of the lanes' heads; round q's winner
            // becomes path q
#pragma unroll
            for (int q = 0; q < L; q++) {
                unsigned bk = key[0], bc = cid[0];
#pragma unroll
                for (int d = 1; d < DL; d <<= 1) {
                    const unsigned ok = __shfl_xor_sync(kFull, bk, d);
                    const unsigned oc = __shfl_xor_sync(kFull, bc, d);
                    const bool take = ok < bk || (ok == bk && oc < bc);
                    bk = take ? ok : bk;
                    bc = take ? oc : bc;
                }
                if (c.l == q) {
                    mkey = bk;
                    mcid = bc;
                }
                if (q + 1 < L && cid[0] == bc) {  // the owner pops its head (ids are unique)
#pragma unroll
                    for (int j = 0; j + 1 < T; j++) {
                        key[j] = key[j + 1];
                        cid[j] = cid[j + 1];
                    }
                    key[T - 1] = 0xffffffffu;  // an exhausted list offers nothing
                    cid[T - 1] = 0xffffffffu;
                }
            }
        }
        const int par = (int)(mcid >> (S + 1)) & (L - 1);
        const int k = (int)(mcid >> 1) & (NS - 1);
        const unsigned neg = mcid & 1u;
        p.pm = ordered_float(mkey);
        list_step<OFF, PC>(c, p, par, pend);
        // decided bits x_j = <k, j> xor sign over the span
        auto pattern = [&](int kk, int wd) {
            unsigned pat = 0;
#pragma unroll
            for (int t = 0; t < 5; t++) {
                const unsigned mt = t == 0 ? 0xAAAAAAAAu : t == 1 ? 0xCCCCCCCCu : t == 2 ? 0xF0F0F0F0u
                                   : t == 3 ? 0xFF00FF00u : 0xFFFF0000u;
                if (t < S && ((kk >> t) & 1)) pat ^= mt;
            }
            if ((__popc((unsigned)(kk >> 5) & (unsigned)wd) & 1) ^ neg) pat = ~pat;
            return pat;
        };
        if constexpr (NS >= 32) {
#pragma unroll
            for (int wd = 0; wd < NS / 32; wd++) p.x[OFF / 32 + wd] = pattern(k, wd);
        } else {
            put_bits<OFF, NS>(p, pattern(k, 0));
        }
        return par;  // the parent path (this lane's new path descends from it)
    }

    // --------------------------------------------------------------- SPCL leaf ---
    // RM(2, 3) node (Eqs. (2)-(6)): parity, PM += p |alpha_lrb|, then tau = min(L, 7) list
    // splits on the next least reliable positions (flip cost |alpha_i| + (1-2p)|alpha_lrb|, each
    // a 2L -> L selection by (PM, 2 path + flip)); the least reliable bit restores even parity.
    template <int OFF, int NS>
    __device__ __forceinline__ static void spc_leaf(const Ctx& c, Path& p, float (&as)[NS / G]) {
        constexpr int TAU = cmin(L, NS - 1);
        // the node's 8 LLRs in every lane of the path (both lanes of a path then hold the same
        // state and take the same decisions; shuffles read a path's lane g = 0)
        float a[NS];
        if constexpr (G == 1) {
#pragma unroll
            for (int i = 0; i < NS; i++) a[i] = as[i];
        } else {
#pragma unroll
            for (int e = 0; e < NS / G; e++) {
                const float o = __shfl_xor_sync(kFull, as[e], 1);
                a[G * e] = c.g ? o : as[e];
                a[G * e + 1] = c.g ? as[e] : o;
            }
        }
        // reliability order (|alpha|, position) ascending: Batcher's odd-even merge sort network
        float sv[NS];
        int sp[NS];
#pragma unroll
        for (int i = 0; i < NS; i++) {
            sv[i] = fabsf(a[i]);
            sp[i] = i;
        }
        auto cx = [&](int i, int j) {  // order entries i < j
            const bool sw = sv[j] < sv[i] || (sv[j] == sv[i] && sp[j] < sp[i]);
            const float tv = sv[i];
            const int tp = sp[i];
            sv[i] = sw ? sv[j] : sv[i];
            sp[i] = sw ? sp[j] : sp[i];
            sv[j] = sw ? tv : sv[j];
            sp[j] = sw ? tp : sp[j];
        };
        constexpr OddEvenMergeNet<NS> net;
        static_assert(net.n <= OddEvenMergeNet<NS>::kMax, "comparators");
#pragma unroll
        for (int t = 0; t < net.n; t++) cx(net.lo[t], net.hi[t]);
        const int o0 = sp[0];
        const float lrb = sv[0];
        float rel[TAU];
        int pos[TAU];
#pragma unroll
        for (int t = 0; t < TAU; t++) {
            rel[t] = sv[1 + t];
            pos[t] = sp[1 + t];
        }
        unsigned hd = 0;
#pragma unroll
        for (int i = 0; i < NS; i++) hd |= (a[i] < 0.f ? 1u : 0u) << i;
        int par = __popc(hd) & 1;
        float pm = p.pm + (par ? lrb : 0.f);  // Eq. (3)
        unsigned flip = 0;
        int orig = c.l;
#pragma unroll 1
        for (int t = 1; t <= TAU; t++) {
            // the split position and the LRB belong to the path's SPC-entry ancestor `orig`
            const int so = c.dbase + G * orig;
            const float r_o = __shfl_sync(kFull, rel[0], so);
            const int itp = __shfl_sync(kFull, pos[0], so);
            const float lrb_o = __shfl_sync(kFull, lrb, so);
            const float pflip = pm + r_o + (par ? -lrb_o : lrb_o);  // Eq. (4)
            // ranks of this path's candidates 2l (keep) and 2l + 1 (flip) among the 2L
            int rk = 0, rf = 0;
#pragma unroll
            for (int l2 = 0; l2 < L; l2++) {
                const float k2 = __shfl_sync(kFull, pm, c.dbase + G * l2);
                const float f2 = __shfl_sync(kFull, pflip, c.dbase + G * l2);
                rk += (k2 < pm) || (k2 == pm && l2 < c.l);
                rk += (f2 < pm) || (f2 == pm && l2 < c.l);
                rf += (k2 < pflip) || (k2 == pflip && l2 <= c.l);
                rf += (f2 < pflip) || (f2 == pflip && l2 < c.l);
            }
            // the candidate of rank q becomes path q
            if (c.g == 0 && rk < L) c.sel[c.dbase + rk] = (uint8_t)(2 * c.l);
            if (c.g == 0 && rf < L) c.sel[c.dbase + rf] = (uint8_t)(2 * c.l + 1);
            __syncwarp();
            const int mysrc = c.sel[c.dbase + c.l];
            __syncwarp();
            const int sl = c.dbase + G * ((mysrc >> 1) & (L - 1));
            const bool fl = mysrc & 1;
            const float n_kpm = __shfl_sync(kFull, pm, sl);
            const float n_fpm = __shfl_sync(kFull, pflip, sl);
            const unsigned packed = __shfl_sync(kFull, (unsigned)orig | ((unsigned)par << 8) | ((unsigned)itp << 16), sl);
            const unsigned n_flip = __shfl_sync(kFull, flip, sl);
            pm = fl ? n_fpm : n_kpm;
            orig = (int)(packed & 0xffu) & (L - 1);
            const int n_it = (int)(packed >> 16) & (NS - 1);
            flip = fl ? (n_flip ^ (1u << n_it)) : n_flip;  // Eq. (5)
            par = (int)((packed >> 8) & 1u) ^ (fl ? 1 : 0);
#pragma unroll
            for (int k = 0; k + 1 < TAU; k++) {
                rel[k] = rel[k + 1];
                pos[k] = pos[k + 1];
            }
        }
        const int so = c.dbase + G * orig;
        const unsigned hd_o = __shfl_sync(kFull, hd, so);
        const int lo0 = __shfl_sync(kFull, o0, so) & (NS - 1);
        constexpr unsigned span = (1u << NS) - 1u;
        unsigned x = ((hd_o ^ flip) & span) & ~(1u << lo0);
        x |= (unsigned)(__popc(x) & 1) << lo0;  // Eq. (6)
        p.pm = pm;
        float none[1];
        list_step<OFF, 0>(c, p, orig, none);
        put_bits<OFF, NS>(p, x);
    }

    // ------------------------------------------------------------- tree walk ---
    // RM(2, S) node off the root (not permuted), LLRs `a`, at span offset OFF
    template <int S, int OFF, bool COL = (R == 2 && PEND_SMEM && S == M - 1)>
    __device__ __forceinline__ static void node2(const Ctx& c, Path& p, float (&a)[(1 << S) / G]) {
        if constexpr (S == 3) {
            spc_leaf<OFF, 8>(c, p, a);
        } else {
            constexpr int HS = 1 << (S - 1);
            constexpr int VH = HS / G;  // this lane's share of a child's positions
            float ch[VH];
            if constexpr (COL) {
                // park the node's LLRs in this lane's column; the new path reads its parent's
                const int lane = c.dbase + G * c.l + c.g;
                __syncwarp();  // every lane has read the previous decoder's columns
#pragma unroll
                for (int e = 0; e < 2 * VH; e++) c.pend[32 * e + lane] = a[e];
                __syncwarp();
#pragma unroll
                for (int e = 0; e < VH; e++) ch[e] = fminsum(a[e], a[e + VH]);
                float none[1];
                const int par = fht_leaf<S - 1, OFF, 0>(c, p, ch, none);
                const float* pa = c.pend + lane_of(c, par);
#pragma unroll
                for (int e = 0; e < VH; e++) ch[e] = g_fn(pa[32 * e], pa[32 * (e + VH)], bitg(p, OFF + G * e, c.g));
            } else {
#pragma unroll
                for (int e = 0; e < VH; e++) ch[e] = fminsum(a[e], a[e + VH]);
                fht_leaf<S - 1, OFF, 2 * VH>(c, p, ch, a);
#pragma unroll
                for (int e = 0; e < VH; e++) ch[e] = g_fn(a[e], a[e + VH], bitg(p, OFF + G * e, c.g));
            }
            node2<S - 1, OFF + HS>(c, p, ch);
            combine<OFF, HS>(p);
        }
    }

    // RM(2, m-1), the left child of an RM(3, m) root: a permuted node (Algorithm 2). Candidate c'
    // of path l (c' = l, l + L) permutes the path's LLRs, which every path parks in its lane's
    // column: LM in the warp-per-decoder kernel's summation order, the L best candidates, then
    // the new path's LLRs gathered from its source path's column through the candidate's map;
    // after the subtree the span is un-permuted through the inverse map.
    template <int S>
    __device__ __forceinline__ static void node2p(const Ctx& c, Path& p, float (&a)[1 << S]) {
        static_assert(R == 3 && G == 1 && S == M - 1, "the permuted child of an RM(3, m) root");
        constexpr int NS = 1 << S;
        constexpr int HALF = NS / 2;
        const int lane = c.dbase + c.l;
        __syncwarp();  // every lane has read the previous decoder's columns
#pragma unroll
        for (int e = 0; e < NS; e++) c.pend[32 * e + lane] = a[e];
        __syncwarp();
        const uint16_t* lrec = c.rec + 2 * L * kRec;  // this level's 2L records
        const float* mine_col = c.pend + lane;
        constexpr int V = HALF < 32 ? HALF : 32;
        float lm[2];
#pragma unroll
        for (int q = 0; q < 2; q++) {
            const uint16_t* r = lrec + (c.l + q * L) * kRec;
            const int am = r[S - 1];
            const int hm = ~((1 << (31 - __clz(am))) - 1);
            float acc[V];
#pragma unroll
            for (int lv = 0; lv < V; lv++) {
                float sum = 0.f;
#pragma unroll
                for (int t = 0; t < (HALF + 31) / 32; t++) {
                    const int jp = lv + 32 * t;
                    const int j = jp + (jp & hm);
                    sum += fminf(fabsf(mine_col[32 * j]), fabsf(mine_col[32 * (j ^ am)]));
                }
                acc[lv] = sum;
            }
#pragma unroll
            for (int d = 16; d >= 1; d >>= 1)
#pragma unroll
                for (int lv = 0; lv < d; lv++)
                    if (lv + d < V) acc[lv] += acc[lv + d];
            lm[q] = acc[0];
        }
        const int cq = pick_by_rank(c, lm);
        // the new path takes its source path's state, and its LLRs through pi_c: a'[i] = a_src[pi(i)]
        const int src = c.dbase + (cq & (L - 1));
        p.pm = __shfl_sync(kFull, p.pm, src);
        p.rootc = __shfl_sync(kFull, p.rootc, src);
        p.selc = cq;
        {
            const uint16_t* r = lrec + cq * kRec;
            int pc[S];
#pragma unroll
            for (int t = 0; t < S; t++) pc[t] = r[t];
            const float* scol = c.pend + src;
            int sv = r[10];
#pragma unroll
            for (int n = 0; n < NS; n++) {
                if (n) sv ^= pc[ctz7(n)];
                a[n ^ (n >> 1)] = scol[32 * sv];
            }
        }
        node2<S, 0, true>(c, p, a);
        // undo pi on the span: x[j] = x'[pi^-1(j)], through the stored inverse map
        {
            const uint16_t* ri = c.rinv + (2 * L + p.selc) * kRec;
            int ic[S];
#pragma unroll
            for (int t = 0; t < S; t++) ic[t] = ri[t];
            constexpr int SW = (NS + 31) / 32;
            uint32_t nx[SW];
#pragma unroll
            for (int w = 0; w < SW; w++) nx[w] = 0;
            int tv = ri[10];
#pragma unroll
            for (int n = 0; n < NS; n++) {
                if (n) tv ^= ic[ctz7(n)];
                const int jj = n ^ (n >> 1);
                const uint32_t word = (SW > 1 && (tv >> 5)) ? p.x[SW > 1 ? 1 : 0] : p.x[0];
                nx[jj >> 5] |= ((word >> (tv & 31)) & 1u) << (jj & 31);
            }
            if constexpr (NS >= 32) {
#pragma unroll
                for (int w = 0; w < SW; w++) p.x[w] = nx[w];
            } else {
                constexpr uint32_t mask = (1u << NS) - 1u;
                p.x[0] = (p.x[0] & ~mask) | nx[0];
            }
        }
    }

    // RM(3, S) node on the right spine of an RM(3, m) tree, LLRs `a`, at span offset OFF: its
    // LLRs wait in the lane's column of level S while its left child RM(2, S-1) runs; paths
    // created meanwhile inherit the lane whose column holds their ancestor's LLRs
    template <int S, int OFF>
    __device__ __forceinline__ static void node3(const Ctx& c, Path& p, float (&a)[1 << S]) {
        if constexpr (S == 4) {
            spc_leaf<OFF, 16>(c, p, a);
        } else {
            constexpr int HS = 1 << (S - 1);
            constexpr int LV = S == M - 1 ? 0 : 1;
            static_assert(S == M - 1 || (S == M - 2 && COL1 > 0), "a column per pending level");
            float* colbase = c.pend + (LV == 0 ? 0 : H * 32);
            const int lane = c.dbase + c.l;
            __syncwarp();
#pragma unroll
            for (int e = 0; e < 2 * HS; e++) colbase[32 * e + lane] = a[e];
            __syncwarp();
            p.own[LV] = lane;
            float ch[HS];
#pragma unroll
            for (int e = 0; e < HS; e++) ch[e] = fminsum(a[e], a[e + HS]);
            node2<S - 1, OFF, false>(c, p, ch);
            const float* pa = colbase + p.own[LV];
#pragma unroll
            for (int e = 0; e < HS; e++) ch[e] = g_fn(pa[32 * e], pa[32 * (e + HS)], bit(p, OFF + e));
            node3<S - 1, OFF + HS>(c, p, ch);
            combine<OFF, HS>(p);
        }
    }

    // The root's 2L candidates (Algorithm 2's permutation decoding): candidate c permutes y
    // through its composed record; LM_c = sum over the pairs {j, j ^ a} of min(|y_j|, |y_{j^a}|),
    // a the image of the top index bit, summed as the warp-per-decoder kernel's lanes and warp
    // reduction do. Returns this path's candidate: the one of rank l by (LM desc, c asc).
    __device__ __forceinline__ static int select_root(const Ctx& c) {
        constexpr int V = H < 32 ? H : 32;  // lanes of that kernel holding pairs
        static_assert(V % G == 0, "its lanes split evenly over a path's lanes");
        constexpr int VL = V / G;            // of them, the ones this lane sums: lv = G u + g
        float lm[2];
#pragma unroll
        for (int q = 0; q < 2; q++) {
            const uint16_t* r = c.rec + (c.l + q * L) * kRec;
            const int a = r[M - 1];
            const int hm = ~((1 << (31 - __clz(a))) - 1);  // index bits at and above bit msb(a)
            float acc[VL];
#pragma unroll
            for (int u = 0; u < VL; u++) {
                float s = 0.f;
#pragma unroll
                for (int t = 0; t < (H + 31) / 32; t++) {
                    const int jp = G * u + c.g + 32 * t;  // the pair's representative: bit msb(a) clear
                    const int j = jp + (jp & hm);
                    s += fminf(fabsf(c.y[j]), fabsf(c.y[j ^ a]));
                }
                acc[u] = s;
            }
            // that kernel's warp sum, d = 16, 8, ..., 1: the steps d >= G within this lane, then
            // (G = 2) d = 1 between the path's two lanes
#pragma unroll
            for (int d = 16; d >= G; d >>= 1)
#pragma unroll
                for (int u = 0; u < d / G; u++)
                    if (u + d / G < VL) acc[u] += acc[u + d / G];
            if constexpr (G == 2) acc[0] += __shfl_xor_sync(kFull, acc[0], 1);
            lm[q] = acc[0];
        }
        return pick_by_rank(c, lm);
    }

    // The candidate of rank l among the decoder's 2L by (LM descending, c ascending), where
    // lane l of the path holds LM of candidates l and l + L.
    __device__ __forceinline__ static int pick_by_rank(const Ctx& c, const float (&lm)[2]) {
        if constexpr (L == 1) {
            return (lm[1] > lm[0]) ? 1 : 0;
        } else {
            int rk[2] = {0, 0};
#pragma unroll
            for (int l2 = 0; l2 < L; l2++) {
#pragma unroll
                for (int q2 = 0; q2 < 2; q2++) {
                    const float o = __shfl_sync(kFull, lm[q2], c.dbase + G * l2);
                    const int c2 = l2 + q2 * L;
#pragma unroll
                    for (int q = 0; q < 2; q++) {
                        const int cc = c.l + q * L;
                        rk[q] += (o > lm[q]) || (o == lm[q] && c2 < cc);
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < 2; q++)
                if (c.g == 0 && rk[q] < L) c.sel[c.dbase + rk[q]] = (uint8_t)(c.l + q * L);
            __syncwarp();
            const int mine = c.sel[c.dbase + c.l] & (2 * L - 1);
            __syncwarp();
            return mine;
        }
    }

    // One decoder (Algorithm 2 from the root). Path 0 ends as the decoder's best path, its
    // bits combined below the root.
    __device__ __forceinline__ static void run(const Ctx& c, Path& p) {
        p.rootc = select_root(c);
        p.pm = (c.single && (p.rootc & (L - 1)) != 0) ? __int_as_float(0x7f800000) : 0.f;
        p.selc = 0;
        p.own[0] = p.own[1] = c.dbase + G * c.l + c.g;
#pragma unroll
        for (int w = 0; w < NW; w++) p.x[w] = 0;
        constexpr int VH = H / G;  // this lane's positions of a root child: G e + g
        constexpr int LG = G == 2 ? 1 : 0;
        float a[VH];
        int col[M - 1];
        int sb, sa;
        auto load_rec = [&]() {
            const uint16_t* r = c.rec + p.rootc * kRec;
#pragma unroll
            for (int t = 0; t < M - 1; t++) col[t] = r[t];
            sa = r[M - 1];
            sb = r[10] ^ ((G == 2 && c.g) ? col[0] : 0);  // the image of position g
        };
        // f: left child RM(r-1, m-1) from y through the path's root permutation, this lane's
        // positions in Gray-code order of e (one XOR per position)
        load_rec();
        {
            int s = sb;
#pragma unroll
            for (int n = 0; n < VH; n++) {
                if (n) s ^= col[LG + ctz7(n)];
                const int e = n ^ (n >> 1);
                a[e] = fminsum(c.y[s], c.y[s ^ sa]);
            }
        }
        if constexpr (R == 2) {
            float none[1];
            fht_leaf<M - 1, 0, 0>(c, p, a, none);
        } else {
            node2p<M - 1>(c, p, a);
        }
        // g: right child RM(r, m-1) from y through the (possibly new) path's permutation
        load_rec();
        {
            int s = sb;
#pragma unroll
            for (int n = 0; n < VH; n++) {
                if (n) s ^= col[LG + ctz7(n)];
                const int e = n ^ (n >> 1);
                a[e] = g_fn(c.y[s], c.y[s ^ sa], bitg(p, G * e, c.g));
            }
        }
        if constexpr (R == 2) node2<M - 1, H>(c, p, a);
        else node3<M - 1, H>(c, p, a);
    }
};

// Decodes the frames of the job, one warp per 32 / FW frames (see Ppt).
// Words of a warp's reduction slots: per staged frame its best decoder's metric key, index and
// metric, and the decoder's codeword (32 / FW frames of 3 + N / 32 words; at most 128 words).
constexpr int kPptSlotWords = 128;

// Resident CTAs of 4 warps the register budget is sized for: 168 registers per thread for
// m >= 6 and for RM(3, m) (measured on RM(2,7) P=8 L=4: 79.0 M frames/s, against 71.0 M at 128
// registers, where the largest leaf spills), 102 for shorter RM(2, m) codes.
__host__ __device__ constexpr int ppt_min_blocks(int m, int r) { return (m >= 6 || r == 3) ? 3 : 5; }

template <int M, int R, int L>
__global__ void __launch_bounds__(128, ppt_min_blocks(M, R)) ppt_kernel(LaunchArgs a) {
    using D = Ppt<M, R, L>;
    constexpr int N = D::N, NW = D::NW, NREC = D::NREC, DL = D::DL;
    constexpr int K = 1 + M + M * (M - 1) / 2 + (R == 3 ? M * (M - 1) * (M - 2) / 6 : 0);  // of RM(r, m)
    constexpr int KW = (K + 31) / 32;
    extern __shared__ __align__(16) uint8_t smem[];
    const int FW = ppt_frame_lanes(M, L, a.P);
    const int FPW = 32 / FW;
    const int YS = ppt_frame_stride(M, FPW);  // floats per staged frame
    const int W = blockDim.x >> 5;
    // shared memory: the P decoders' maps and inverse maps as in the device table, the
    // information positions, the staged frames' LLRs, then per warp its level-(m-1) columns, a
    // selection scratch and its reduction slots
    const int rec_elems = a.P * 2 * NREC * kRec;
    uint16_t* s_rec = reinterpret_cast<uint16_t*>(smem);
    uint16_t* s_info = s_rec + rec_elems;
    const int tables = ((rec_elems * 2 + K * 2) + 15) / 16 * 16;
    float* s_y = reinterpret_cast<float*>(smem + tables);
    const int ybytes = ((FPW * YS * 4) + 15) / 16 * 16;
    const int warp_bytes = D::PEND_FLOATS * 4 + 32 + kPptSlotWords * 4;
    for (int i = threadIdx.x; i < rec_elems; i += blockDim.x) s_rec[i] = a.recs[i];
    for (int i = threadIdx.x; i < K; i += blockDim.x) s_info[i] = a.info[i];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint8_t* wbase = smem + tables + ybytes;
    float* s_pend = reinterpret_cast<float*>(wbase + warp * warp_bytes);
    uint8_t* s_sel = wbase + warp * warp_bytes + D::PEND_FLOATS * 4;
    auto slots = [&](int w) { return reinterpret_cast<uint32_t*>(wbase + w * warp_bytes + D::PEND_FLOATS * 4 + 32); };
    const int grp = lane / FW, j = lane % FW, gbase = grp * FW;
    const int DPB = FW / DL;                // decoders per batch
    const int NB = (a.P + DPB - 1) / DPB;  // batches per frame
    const int ds = j / DL;
    typename D::Ctx c;
    c.y = s_y + grp * YS;
    c.sel = s_sel;
    c.pend = s_pend;
    c.dbase = gbase + ds * DL;
    c.l = (j % DL) / D::G;
    c.g = j % D::G;
    c.single = a.single_start != 0;
    c.int8 = a.dtype == IN_I8;
    const unsigned gmask = FW == 32 ? 0xffffffffu : ((1u << FW) - 1u);
    const size_t eb = a.dtype == IN_F32 ? 4 : (a.dtype == IN_I8 ? 1 : 2);
    const int64_t nblk = (a.n_frames + FPW - 1) / FPW;
    for (int64_t fb = blockIdx.x; fb < nblk; fb += gridDim.x) {
        const int64_t f0 = fb * FPW;
        __syncthreads();  // the previous frames' LLRs and slots are no longer read
        // the FPW frames' LLRs (contiguous), 16 bytes per load, widened to float
        {
            const int chunks = (int)(FPW * N * eb / 16);
            const int per = (int)(16 / eb);  // values per chunk
            const uint4* src = reinterpret_cast<const uint4*>(static_cast<const uint8_t*>(a.llr) + f0 * N * eb);
            for (int i = threadIdx.x; i < chunks; i += blockDim.x) {
                if (f0 + (int64_t)(i * per) / N >= a.n_frames) continue;
                const uint4 q = src[i];
                const uint32_t wv[4] = {q.x, q.y, q.z, q.w};
                const int q0 = i * per;  // first value of the chunk; chunks never straddle frames
                float4* dst = reinterpret_cast<float4*>(s_y + (q0 / N) * YS + q0 % N);
                if (a.dtype == IN_F32) {
                    dst[0] = make_float4(__uint_as_float(wv[0]), __uint_as_float(wv[1]), __uint_as_float(wv[2]),
                                         __uint_as_float(wv[3]));
                } else if (a.dtype == IN_I8) {
#pragma unroll
                    for (int b = 0; b < 4; b++)
                        dst[b] = make_float4((float)((int32_t)(wv[b] << 24) >> 24), (float)((int32_t)(wv[b] << 16) >> 24),
                                             (float)((int32_t)(wv[b] << 8) >> 24), (float)((int32_t)wv[b] >> 24));
                } else if (a.dtype == IN_F16) {
                    auto h = [](uint32_t w, int hi) {
                        return __half2float(__ushort_as_half((unsigned short)(hi ? (w >> 16) : (w & 0xffffu))));
                    };
#pragma unroll
                    for (int b = 0; b < 2; b++)
                        dst[b] = make_float4(h(wv[2 * b], 0), h(wv[2 * b], 1), h(wv[2 * b + 1], 0), h(wv[2 * b + 1], 1));
                } else {
                    float v8[8];
#pragma unroll
                    for (int b = 0; b < 4; b++) {
                        v8[2 * b] = fminf(fmaxf((float)((int32_t)(wv[b] << 16) >> 16), -a.qclamp), a.qclamp);
                        v8[2 * b + 1] = fminf(fmaxf((float)((int32_t)wv[b] >> 16), -a.qclamp), a.qclamp);
                    }
                    dst[0] = make_float4(v8[0], v8[1], v8[2], v8[3]);
                    dst[1] = make_float4(v8[4], v8[5], v8[6], v8[7]);
                }
            }
        }
        __syncthreads();
        const int64_t f = f0 + grp;
        // this warp's best decoder over its batches (batches in increasing order: strict <
        // keeps the earliest of equal metrics)
        unsigned best_key = 0xffffffffu;
        int best_d = 1 << 30;
        float best_pm = 0.f;
        uint32_t cw[NW];
#pragma unroll
        for (int w = 0; w < NW; w++) cw[w] = 0;
        for (int bt = warp; bt < NB; bt += W) {
            const int b0 = bt * DPB;
            const int d = b0 + ds;
            const bool dvalid = d < a.P;
            const int dd = dvalid ? d : a.P - 1;
            c.rec = s_rec + dd * 2 * NREC * kRec;
            c.rinv = c.rec + NREC * kRec;
            typename D::Path p;
            D::run(c, p);
            // Algorithm 5 over the batch: the smallest metric (NaN last), earlier decoders
            // first; lanes of path 0 hold each decoder's best path
            const float v = p.pm == p.pm ? p.pm : __int_as_float(0x7f800000);
            unsigned bk = dvalid ? ordered_bits(v) : 0xffffffffu;
            unsigned bd = (unsigned)ds;
            for (int dl = DL; dl < FW; dl <<= 1) {
                const unsigned ok = __shfl_xor_sync(kFull, bk, dl);
                const unsigned od = __shfl_xor_sync(kFull, bd, dl);
                const bool take = ok < bk || (ok == bk && od < bd);
                bk = take ? ok : bk;
                bd = take ? od : bd;
            }
            bk = __shfl_sync(kFull, bk, gbase);
            bd = __shfl_sync(kFull, bd, gbase);
            const int wl = gbase + (int)bd * DL;
            uint32_t xw[NW];
#pragma unroll
            for (int w = 0; w < NW; w++) xw[w] = __shfl_sync(kFull, p.x[w], wl);
            const int wc = __shfl_sync(kFull, p.rootc, wl);
            const float wpm = __shfl_sync(kFull, p.pm, wl);
            // root combine, then x[sigma(i)] = x'[i]: bit q of the codeword is bit sigma^-1(q)
            // of the permuted word, read through the stored inverse map; lane j of the group
            // takes positions j + FW t (every lane of the warp runs this: the ballots need them)
            if constexpr (D::H >= 32) {
#pragma unroll
                for (int w = 0; w < NW / 2; w++) xw[w] ^= xw[w + NW / 2];
            } else {
                xw[0] ^= (xw[0] >> D::H) & ((1u << D::H) - 1u);
            }
            const int dw = b0 + (int)bd;
            const uint16_t* ri = s_rec + (dw * 2 + 1) * NREC * kRec + wc * kRec;
            uint32_t nw[NW];
#pragma unroll
            for (int w = 0; w < NW; w++) {  // word w: FW positions per ballot
                nw[w] = 0;
                for (int o = 0; o < 32 && 32 * w + o < N; o += FW) {
                    const int q = 32 * w + o + j;
                    unsigned b = 0;
                    if (q < N) {
                        const int sp = ga_apply(ri, M, q);
                        b = (pick_word(xw, sp >> 5) >> (sp & 31)) & 1u;
                    }
                    nw[w] |= ((__ballot_sync(kFull, b) >> gbase) & gmask) << o;
                }
            }
            if (bk < best_key || bt == warp) {  // strict: earlier decoders win ties
#pragma unroll
                for (int w = 0; w < NW; w++) cw[w] = nw[w];
                best_key = bk;
                best_d = dw;
                best_pm = wpm == wpm ? wpm : __int_as_float(0x7f800000);
            }
        }
        // Algorithm 5 across the warps: the smallest (metric key, decoder) per frame
        if (W > 1) {
            uint32_t* sl = slots(warp) + grp * (3 + NW);
            if (j == 0) {
                sl[0] = best_key;
                sl[1] = (uint32_t)best_d;
                sl[2] = __float_as_uint(best_pm);
            }
            if (j < NW) sl[3 + j] = pick_word(cw, j);
            __syncthreads();
            if (warp != 0) continue;  // warp 0 writes the CTA's frames
            int bw = 0;
            unsigned bkey = 0xffffffffu;
            int bdec = 1 << 30;
            for (int w2 = 0; w2 < W; w2++) {
                const uint32_t* o = slots(w2) + grp * (3 + NW);
                const unsigned ok = o[0];
                const int od = (int)o[1];
                if (ok < bkey || (ok == bkey && od < bdec)) {
                    bkey = ok;
                    bdec = od;
                    bw = w2;
                }
            }
            const uint32_t* o = slots(bw) + grp * (3 + NW);
            best_d = (int)o[1];
            best_pm = __uint_as_float(o[2]);
#pragma unroll
            for (int w = 0; w < NW; w++) cw[w] = o[3 + w];
        }
        // outputs: codeword, metric, winner, and u = x G^{(x)m} at the information positions
        const bool fvalid = f < a.n_frames;
        if (fvalid && a.cw_out && j < NW) a.cw_out[f * NW + j] = pick_word(cw, j);
        if (fvalid && j == 0) {
            if (a.pm_out) a.pm_out[f] = best_pm;
            if (a.best_out) a.best_out[f] = best_d;
        }
        uint32_t u[NW];
#pragma unroll
        for (int w = 0; w < NW; w++) {
            unsigned v = cw[w];
            v ^= (v >> 1) & 0x55555555u;
            v ^= (v >> 2) & 0x33333333u;
            v ^= (v >> 4) & 0x0F0F0F0Fu;
            v ^= (v >> 8) & 0x00FF00FFu;
            if (M > 4) v ^= (v >> 16) & 0x0000FFFFu;
            u[w] = v;
        }
#pragma unroll
        for (int t = 5; t < M; t++) {
            constexpr int one = 1;
            const int dd = one << (t - 5);
#pragma unroll
            for (int w = 0; w < NW; w++)
                if (!(w & dd)) u[w] ^= u[w | dd];
        }
        uint32_t iw[KW];
#pragma unroll
        for (int w = 0; w < KW; w++) {  // information word w: FW positions per ballot
            iw[w] = 0;
            for (int o = 0; o < 32 && 32 * w + o < K; o += FW) {
                const int q = 32 * w + o + j;
                unsigned b = 0;
                if (q < K) {
                    const int pos = s_info[q];
                    b = (pick_word(u, pos >> 5) >> (pos & 31)) & 1u;
                }
                iw[w] |= ((__ballot_sync(kFull, b) >> gbase) & gmask) << o;
            }
        }
        if (fvalid && j < KW) a.info_out[f * KW + j] = pick_word(iw, j);
    }
}

}  // namespace rmdec_dev
