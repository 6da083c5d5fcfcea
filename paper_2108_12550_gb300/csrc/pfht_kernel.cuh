// p-FHT-FSCL-L-M decoding kernel for RM(r, m) on sm_103a.
//
// Method: Doan, Hashemi, Gross, arXiv 2108.12550 — Algorithm 2 (permuted recursion),
// Algorithms 3-4 with Eq. (8) (FHTL on RM(1, s) nodes), Eqs. (2)-(6) (SPCL on RM(s-1, s)
// nodes) and Algorithm 5 (best of P decoders).
//
// Execution model. A CTA owns one frame at a time (persistent loop over frames). Its W warps
// share the frame's LLRs in shared memory and split the P decoders round-robin; a warp runs
// one decoder with all L list paths at once, and the warps of a CTA run their decoders in
// lockstep (block barriers at every leaf and after every round; see Decoder). The decoding tree is expanded at compile time
// (template recursion over (r_v, m_v, span offset)), so every node's size, lane mapping and
// register arrays are static. Per warp, shared memory holds one LLR buffer per tree level
// with L slots; list reselection never copies LLRs: each path keeps, per pending ancestor
// level, the slot index of its ancestor's LLRs (shuffled from the parent lane on every list
// step). Decided bits of finished nodes sit in a per-path packed bit buffer (double
// buffered; a list step copies only the words left of the current node); permuted nodes
// un-permute them by gathering through the inverse maps the host stores with the maps.
//
// Exactness: the arithmetic is add, subtract, min, abs, negate, compare and multiply by 1/2.
// On integer-valued LLRs below 2^24 / 2^m every intermediate value is an exactly
// represented integer, so the integer input types decode bit-exactly.
#pragma once

#include <cstdint>
#include <type_traits>

#include <cuda_fp16.h>

namespace rmdec_dev {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kRec = 11;      // uint16 per permutation record: [c_0..c_9, b]
constexpr int kMaxWarps = 20; // widest pfht_kernel CTA (its register budget: 96 per thread)

enum InType { IN_F32 = 0, IN_I8 = 1, IN_F16 = 2, IN_I16 = 3 };

__host__ __device__ constexpr int cmin(int a, int b) { return a < b ? a : b; }
__host__ __device__ constexpr int cilog2(int x) { return x <= 1 ? 0 : 1 + cilog2(x >> 1); }

struct LaunchArgs {
    const void* llr;
    int dtype;
    float qclamp;  // |code| clamp for I16 inputs
    int64_t n_frames;
    int P;
    const uint16_t* recs;  // device records: per decoder NREC maps, then their NREC inverses
    const uint16_t* info;  // K information positions
    int K;
    uint32_t* info_out;  // [F][ceil(K/32)]
    uint32_t* cw_out;    // [F][ceil(N/32)] or null
    float* pm_out;       // [F] or null
    int32_t* best_out;   // [F] or null
    int single_start;    // one live initial path (FHT-FSCL without permutations)
};

// Shared-memory layout of one decoder configuration.
template <int M, int R, int L>
struct Cfg {
    static constexpr int N = 1 << M;
    static constexpr int NW = N >= 32 ? N / 32 : 1;
    static constexpr int NLEV = R - 1;           // permuted nodes: levels M, M-1, ..., M-R+2
    static constexpr int NREC = 2 * L * NLEV;    // candidate permutations per decoder (device
                                                 // tables: NREC maps, then their NREC inverses)
    static constexpr int MIN_DEEP = M - R + 2;   // lowest permuted level

    static __host__ __device__ constexpr int lanes(int s) { return cmin(32 / L, 1 << s); }
    static __host__ __device__ constexpr int stride(int s) {
        return (1 << s) + (((1 << s) >= 32) ? lanes(s) : 0);
    }
    static __host__ __device__ constexpr int lvl_floats(int s) { return L * stride(s); }
    static __host__ __device__ constexpr int lvl_off(int s) {  // main buffers, levels 2..M-1
        int o = 0;
        for (int t = 2; t < s; t++) o += lvl_floats(t);
        return o;
    }
    static constexpr int MAIN_FLOATS = lvl_off(M);
    static __host__ __device__ constexpr bool deep_perm(int s) { return s < M && s >= MIN_DEEP; }
    static __host__ __device__ constexpr int alt_off(int s) {  // second buffer of permuted levels
        int o = MAIN_FLOATS;
        for (int t = MIN_DEEP; t < s; t++) o += lvl_floats(t);
        return o;
    }
    // LEAN: RM(3, m >= 8), whose warp areas limit the resident warps (shared memory, not
    // registers). The one deeper permuted level (m - 1) then needs no second buffer: its
    // unpermuted LLRs are staged in the lower levels' buffers, which hold nothing yet when
    // the left spine reaches it, and the permuted copies go to the level's own buffer. The
    // permutation maps are read from the device table (L1) instead of block shared memory.
    static constexpr bool LEAN = NLEV == 2 && M >= 8 && lvl_off(MIN_DEEP) >= lvl_floats(MIN_DEEP);
    static constexpr int SMEM_NREC = LEAN ? 0 : NREC;  // maps per decoder in block shared memory
    static constexpr int ALPHA_FLOATS = LEAN ? MAIN_FLOATS : alt_off(M);
    static constexpr int BITS_WORDS = 2 * L * NW;  // double-buffered per-path bit buffers
    // warp area: alpha | bits | xtmp (NW) | best codeword (NW) | spc order (L*32 bytes)
    static constexpr int OFF_BITS = ALPHA_FLOATS * 4;
    static constexpr int OFF_XTMP = OFF_BITS + BITS_WORDS * 4;
    static constexpr int OFF_BEST = OFF_XTMP + NW * 4;
    static constexpr int OFF_SPC = OFF_BEST + NW * 4;
    static constexpr int WARP_BYTES = ((OFF_SPC + L * 32) + 15) / 16 * 16;
    static __host__ constexpr int fixed_bytes(int P, int K, int W);
};

struct Warp {
    float* alpha;       // this warp's LLR buffers
    uint32_t* bits;     // 2 x L x NW
    uint32_t* xtmp;     // NW scratch
    uint32_t* best;     // NW: this warp's best codeword so far
    uint8_t* spc;       // L x 32 SPC order scratch
    const float* y;     // frame LLRs
    const uint16_t* rec;      // this decoder's NREC records (shared memory; LEAN: device table)
    const uint16_t* rec_inv;  // their inverse maps (global memory; read only to un-permute)
    int lane;
    int bsel;           // current bit buffer (warp uniform)
    bool single;        // paths 1..L-1 start inactive (metric +inf)
};

template <int M>
struct PState {
    float pm;            // path metric
    int rootc;           // root candidate (composed permutation) this path descends from
    int slot[M + 1];     // per pending level: slot of the ancestor's LLRs
    int selc[M + 1];     // per deeper permuted level: chosen candidate (pi*)
};

__device__ __forceinline__ float fminsum(float a, float b) {
    // f(a, b) = min(|a|, |b|) sgn(a) sgn(b) (Section II-B). With a zero input the result is
    // a signed zero, which every later step treats as 0 (hard decision 0, |.| = 0).
    const float m = fminf(fabsf(a), fabsf(b));
    return __uint_as_float(__float_as_uint(m) | ((__float_as_uint(a) ^ __float_as_uint(b)) & 0x80000000u));
}
// g(a, b, c) = b + (1 - 2c) a (Section II-B): the sign of a flipped when c = 1
__device__ __forceinline__ float g_fn(float a, float b, unsigned c) {
    return b + __uint_as_float(__float_as_uint(a) ^ (c << 31));
}

// i -> b ^ A v(i) of a record, for i with at most s significant bits
__device__ __forceinline__ int ga_apply(const uint16_t* r, int s, int i) {
    int v = r[10];
#pragma unroll
    for (int t = 0; t < 10; t++)
        if (t < s && ((i >> t) & 1)) v ^= r[t];
    return v;
}
// low part for i = lane + 32 * t: b ^ A (lane), using columns 0..min(5, s)-1
__device__ __forceinline__ int ga_lane_base(const uint16_t* r, int s, int lane) {
    int v = r[10];
#pragma unroll
    for (int t = 0; t < 5; t++)
        if (t < s && ((lane >> t) & 1)) v ^= r[t];
    return v;
}
// high part A (32 t) using columns 5..s-1
__device__ __forceinline__ int ga_hi(const uint16_t* r, int s, int t32) {
    int v = 0;
#pragma unroll
    for (int b = 0; b < 5; b++)
        if (b + 5 < s && ((t32 >> b) & 1)) v ^= r[5 + b];
    return v;
}
__device__ __forceinline__ int insert_zero(int x, int h) {  // insert a 0 bit at position h
    return ((x >> h) << (h + 1)) | (x & ((1 << h) - 1));
}
// Order-preserving map of IEEE single to unsigned (for integer warp reductions) and back.
__device__ __forceinline__ unsigned ordered_bits(float f) {
    const unsigned b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float ordered_float(unsigned u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(kFull, v, d);
    return v;
}

// ------------------------------------------------------ tensor-core Hadamard ---
// D = A B + C on the tensor cores, one warp: A 16x16 and B 16x8 in FP16, C and D in FP32
// (mma.sync m16n8k16). Fragments, with g = lane / 4 and t = lane % 4: A registers hold the
// element pairs (g, 2t..2t+1), (g+8, 2t..2t+1), (g, 2t+8..2t+9), (g+8, 2t+8..2t+9); B registers
// (2t..2t+1, g), (2t+8..2t+9, g); C/D (g, 2t), (g, 2t+1), (g+8, 2t), (g+8, 2t+1).
__device__ __forceinline__ void mma_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ uint32_t pack_half2(float lo, float hi) {
    const __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&h);
}
// entry (i, j) of the Sylvester Hadamard matrix H_16: (-1)^popcount(i & j)
__device__ __forceinline__ float h16(int i, int j) { return (__popc(i & j) & 1) ? -1.f : 1.f; }

// The Walsh-Hadamard spectrum of a vector x of 2^S <= 256 values (S >= 4), in place, on the
// tensor cores: with x read as the R x 16 matrix X[a][b] = x[16 a + b] (R = 2^(S-4)), and
// H_{2^S} = H_R (x) H_16, the spectrum is c[16 p + q] = (H_R X H_16)[p][q]. Both products run as
// m16n8k16 MMAs with H_16 (exact in FP16) on one side: S = H_16 X (X padded to 16 rows with
// zeros; rows p < R of H_16 X are H_R X), then C = S H_16, the FP32 accumulators of S
// rounded to FP16 as the A operand. Inputs enter as FP16 (rounded), sums accumulate in FP32.
template <int S>
__device__ __forceinline__ void tc_hadamard(float* x, int lane) {
    static_assert(S >= 4 && S <= 8, "16 to 256 points");
    constexpr int R = 1 << (S - 4);
    const int g = lane >> 2, t = lane & 3;
    uint32_t ha[4];  // H_16 as the A operand
    ha[0] = pack_half2(h16(g, 2 * t), h16(g, 2 * t + 1));
    ha[1] = pack_half2(h16(g + 8, 2 * t), h16(g + 8, 2 * t + 1));
    ha[2] = pack_half2(h16(g, 2 * t + 8), h16(g, 2 * t + 9));
    ha[3] = pack_half2(h16(g + 8, 2 * t + 8), h16(g + 8, 2 * t + 9));
    auto X = [&](int a, int b) { return a < R ? x[16 * a + b] : 0.f; };
    float sacc[2][4];
#pragma unroll
    for (int h = 0; h < 2; h++) {  // S[:, 8h .. 8h + 7] = H_16 X[:, 8h .. 8h + 7]
        const int col = 8 * h + g;
        const uint32_t b0 = pack_half2(X(2 * t, col), X(2 * t + 1, col));
        const uint32_t b1 = pack_half2(X(2 * t + 8, col), X(2 * t + 9, col));
#pragma unroll
        for (int i = 0; i < 4; i++) sacc[h][i] = 0.f;
        mma_16816(sacc[h], ha, b0, b1);
    }
    // the accumulators of the two column halves of S are its A fragment
    uint32_t sa[4];
    sa[0] = pack_half2(sacc[0][0], sacc[0][1]);
    sa[1] = pack_half2(sacc[0][2], sacc[0][3]);
    sa[2] = pack_half2(sacc[1][0], sacc[1][1]);
    sa[3] = pack_half2(sacc[1][2], sacc[1][3]);
    float cacc[2][4];
#pragma unroll
    for (int h = 0; h < 2; h++) {  // C[:, 8h .. 8h + 7] = S H_16[:, 8h .. 8h + 7]
        const int col = 8 * h + g;
        const uint32_t b0 = pack_half2(h16(2 * t, col), h16(2 * t + 1, col));
        const uint32_t b1 = pack_half2(h16(2 * t + 8, col), h16(2 * t + 9, col));
#pragma unroll
        for (int i = 0; i < 4; i++) cacc[h][i] = 0.f;
        mma_16816(cacc[h], sa, b0, b1);
    }
    __syncwarp();  // every lane has read x
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int q = 8 * h + 2 * t;
        if (g < R) {
            x[16 * g + q] = cacc[h][0];
            x[16 * g + q + 1] = cacc[h][1];
        }
        if (g + 8 < R) {
            x[16 * (g + 8) + q] = cacc[h][2];
            x[16 * (g + 8) + q + 1] = cacc[h][3];
        }
    }
    __syncwarp();
}

// LOCK: every warp of the block runs one decoder per round, so each leaf can start with a
// block barrier that keeps the warps on the same code (see fht_leaf).
// TC: FHTL nodes of 16 to 256 points take their spectra from the tensor cores (tc_hadamard)
// instead of the FP32 butterflies.
template <int M, int R, int L, bool LOCK, bool TC = false>
struct Decoder {
    using C = Cfg<M, R, L>;
    static constexpr int N = C::N;
    static constexpr int NW = C::NW;

    __device__ static uint32_t* bitbuf(Warp& w, int sel, int path) { return w.bits + (sel * L + path) * NW; }

    // ---------------------------------------------------------------- list step ---
    // New path l (lane l < L) descends from `parent`; copies path state and the decided bits
    // left of span offset OFF. PEND: bit s set if the node at level s awaits its right child.
    template <int OFF, unsigned PEND>
    __device__ static void reselect(Warp& w, PState<M>& ps, int parent, float newpm) {
        const int par = w.lane < L ? parent : 0;
        ps.rootc = __shfl_sync(kFull, ps.rootc, par);
#pragma unroll
        for (int s = 2; s < M; s++) {
            if ((PEND >> s) & 1) ps.slot[s] = __shfl_sync(kFull, ps.slot[s], par);
            if (C::deep_perm(s)) ps.selc[s] = __shfl_sync(kFull, ps.selc[s], par);
        }
        ps.pm = newpm;
        constexpr int CW = (OFF + 31) / 32;
        if constexpr (CW > 0) {
            __syncwarp();
            constexpr int TOT = L * CW;
#pragma unroll
            for (int it = 0; it < (TOT + 31) / 32; it++) {
                const int idx = w.lane + 32 * it;
                const int l = idx < TOT ? idx / CW : 0;
                const int pl = __shfl_sync(kFull, par, l);
                if (idx < TOT) {
                    const int wd = idx % CW;
                    bitbuf(w, w.bsel ^ 1, l)[wd] = bitbuf(w, w.bsel, pl)[wd];
                }
            }
            w.bsel ^= 1;
            __syncwarp();
        }
    }

    // Writes `nb` (<= 32) bits `v` of path lane (< L) at span offset OFF (RMW of one word).
    template <int OFF, int NB>
    __device__ static void put_small_bits(Warp& w, unsigned v) {
        static_assert(NB <= 32 && (OFF % NB) == 0, "small span");
        if (w.lane < L) {
            uint32_t* wd = bitbuf(w, w.bsel, w.lane) + OFF / 32;
            const unsigned mask = (NB == 32 ? 0xffffffffu : ((1u << NB) - 1u)) << (OFF % 32);
            *wd = (*wd & ~mask) | ((v << (OFF % 32)) & mask);
        }
        __syncwarp();
    }

    // -------------------------------------------- FHTL selection, long lists ---
    // The same selection as fht_leaf for lists too long to spread over the lanes of a warp
    // (L >= 16 on nodes of 2^S >= 128 points): for each path in turn the whole warp computes its
    // spectrum (position k = lane + 32 e) and its T = min(L, 2^S) candidates of largest |c_k|
    // (ties: smaller k) with PM' = PM_l + (sum|alpha| - |c_k|)/2 (Algorithm 4, Eq. (8)), stored
    // in the buffers of the levels below S (free during a leaf); the L survivors then come from
    // merging the L sorted lists by (PM', l, rank) (Algorithm 3's pool sort by (PM', ordinal)).
    template <int S>
    __device__ static void fht_select_seq(Warp& w, PState<M>& ps, int& my_par, int& my_k, int& my_neg, float& my_pm) {
        constexpr int NS = 1 << S;
        constexpr int EE = NS / 32;
        constexpr int T = cmin(L, NS);
        constexpr int ST = C::stride(S);
        static_assert(EE >= 1 && EE <= 32, "spectrum of 32 to 1024 points");
        static_assert(C::lvl_off(S) >= L * T + (L * T + 1) / 2, "candidate lists fit below the node's level");
        static_assert(NS <= (1 << 15), "codes k << 1 | sign fit 16 bits");
        const float* buf = w.alpha + C::lvl_off(S);
        float* cand_pm = w.alpha;                                             // [L][T]
        uint16_t* cand_code = reinterpret_cast<uint16_t*>(w.alpha + L * T);   // [L][T]: k << 1 | sign
        __syncwarp();
#pragma unroll 1
        for (int l = 0; l < L; l++) {
            float x[EE];
#pragma unroll
            for (int e = 0; e < EE; e++) x[e] = buf[l * ST + w.lane + 32 * e];
            float A = 0.f;
#pragma unroll
            for (int e = 0; e < EE; e++) A += fabsf(x[e]);
            A = warp_sum(A);
#pragma unroll
            for (int h = 1; h < EE; h <<= 1)
#pragma unroll
                for (int e = 0; e < EE; e++)
                    if (!(e & h)) {
                        const float a = x[e], b = x[e + h];
                        x[e] = a + b;
                        x[e + h] = a - b;
                    }
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const float sg = (w.lane & d) ? -1.f : 1.f;
#pragma unroll
                for (int e = 0; e < EE; e++) {
                    const float o = __shfl_xor_sync(kFull, x[e], d);
                    x[e] = fmaf(sg, x[e], o);
                }
            }
            const float pml = __shfl_sync(kFull, ps.pm, l);
            unsigned taken = 0;
#pragma unroll 1
            for (int t = 0; t < T; t++) {
                // the lane's best untaken value (ties: smaller e, i.e. smaller k)
                unsigned key = 0;  // 1 + bits of |c| (|c| >= 0 orders as its bits); 0: none left
                int be = 0;
#pragma unroll
                for (int e = 0; e < EE; e++) {
                    const unsigned kk = ((taken >> e) & 1u) ? 0u : __float_as_uint(fabsf(x[e])) + 1u;
                    if (kk > key) {
                        key = kk;
                        be = e;
                    }
                }
                const unsigned kmax = __reduce_max_sync(kFull, key);
                const unsigned kwin = __reduce_min_sync(kFull, key == kmax ? (unsigned)(w.lane + 32 * be) : 0xffffffffu);
                int neg = 0;
#pragma unroll
                for (int e = 0; e < EE; e++)
                    if (e == be) neg = x[e] < 0.f;
                neg = __shfl_sync(kFull, neg, (int)(kwin & 31u));
                if (w.lane == (int)(kwin & 31u)) taken |= 1u << be;
                if (w.lane == 0) {
                    cand_pm[l * T + t] = pml + 0.5f * (A - __uint_as_float(kmax - 1u));
                    cand_code[l * T + t] = (uint16_t)((kwin << 1) | (unsigned)neg);
                }
            }
        }
        __syncwarp();
        // merge: lane l < L holds the head of path l's list
        int head = 0;
        unsigned hkey = w.lane < L ? ordered_bits(cand_pm[w.lane * T]) : 0xffffffffu;
#pragma unroll 1
        for (int q = 0; q < L; q++) {
            const unsigned kmin = __reduce_min_sync(kFull, hkey);
            const int lw = (int)__reduce_min_sync(kFull, hkey == kmin ? (unsigned)w.lane : 0xffffffffu);
            const int hw = __shfl_sync(kFull, head, lw);
            if (w.lane == q) {
                const int code = cand_code[lw * T + hw];
                my_pm = cand_pm[lw * T + hw];
                my_par = lw;
                my_k = code >> 1;
                my_neg = code & 1;
            }
            if (w.lane == lw) {
                head++;
                hkey = head < T ? ordered_bits(cand_pm[w.lane * T + head]) : 0xffffffffu;
            }
        }
        __syncwarp();  // the lists are read before the caller's list step writes below
    }

    // ------------------------------------------------------------- FHTL leaf ---
    // RM(1, S) node (Algorithms 3-4): per path the Walsh-Hadamard spectrum c of its LLRs,
    // candidates (k, sign c_k) with PM' = PM_l + (sum|alpha| - |c_k|)/2 (Eq. (8)); the L best
    // over all paths by (PM', l, k) survive. Ranking by (PM', l, k) over all L 2^S candidates
    // equals the paper's per-path top-min(L, 2^S) followed by the pool sort with ordinal
    // l*T + rank, because within one path PM' falls as |c_k| rises.
    template <int S, int OFF, unsigned PEND>
    __device__ static void fht_leaf(Warp& w, PState<M>& ps) {
        // The decoders of a block execute the same instruction stream; aligning them at every
        // leaf keeps their warps on the same code, which the tree's instruction footprint
        // (far beyond the instruction caches) rewards. (A barrier under a runtime condition
        // measured 3% slower than this compile-time one.)
        if constexpr (LOCK) __syncthreads();
        constexpr int G = C::lanes(S);
        constexpr int E = (1 << S) / G;
        constexpr int ST = C::stride(S);
        if constexpr (E > 64 || (L >= 16 && E > 32)) {
            // long lists on large nodes: one path at a time with the whole warp
            int my_par = 0, my_k = 0, my_neg = 0;
            float my_pm = 0.f;
            fht_select_seq<S>(w, ps, my_par, my_k, my_neg, my_pm);
            fht_finish<S, OFF, PEND>(w, ps, my_par, my_k, my_neg, my_pm);
            return;
        }
        using Mask = typename std::conditional<(E > 32), unsigned long long, unsigned>::type;
        const float* buf = w.alpha + C::lvl_off(S);
        const bool act = w.lane < L * G;
        const int l = act ? w.lane / G : 0;
        const int g = w.lane % G;
        float v[E];
#pragma unroll
        for (int e = 0; e < E; e++) v[e] = act ? buf[l * ST + g + G * e] : 0.f;
        float A;
        {
            float t[E];
#pragma unroll
            for (int e = 0; e < E; e++) t[e] = fabsf(v[e]);
#pragma unroll
            for (int h = E / 2; h >= 1; h >>= 1)
#pragma unroll
                for (int e = 0; e < h; e++) t[e] += t[e + h];
            A = t[0];
        }
#pragma unroll
        for (int d = 1; d < G; d <<= 1) A += __shfl_xor_sync(kFull, A, d);
        if constexpr (TC && S >= 4 && S <= 8) {
            // spectra of the L paths from the tensor cores, written over the node's LLRs, then
            // read back in this leaf's lane layout
            float* mbuf = w.alpha + C::lvl_off(S);
            __syncwarp();
#pragma unroll 1
            for (int p = 0; p < L; p++) tc_hadamard<S>(mbuf + p * ST, w.lane);
#pragma unroll
            for (int e = 0; e < E; e++) v[e] = act ? buf[l * ST + g + G * e] : 0.f;
        } else {
            // butterflies (u, w) -> (u + w, u - w) over the register bits of the index ...
#pragma unroll
            for (int h = 1; h < E; h <<= 1)
#pragma unroll
                for (int e = 0; e < E; e++)
                    if (!(e & h)) {
                        const float a = v[e], b = v[e + h];
                        v[e] = a + b;
                        v[e + h] = a - b;
                    }
            // ... and over the lane bits
#pragma unroll
            for (int d = 1; d < G; d <<= 1) {
                // lower index: u + w, upper index: u - w, as o + (+-1) v rounded once
                const float sg = (g & d) ? -1.f : 1.f;
#pragma unroll
                for (int e = 0; e < E; e++) {
                    const float o = __shfl_xor_sync(kFull, v[e], d);
                    v[e] = fmaf(sg, v[e], o);
                }
            }
        }
        const float pml = __shfl_sync(kFull, ps.pm, l);
        // Each lane caches its two best candidates by (|c| descending, e ascending) and
        // rescans (excluding taken entries) only when both were taken and another round
        // remains. Rounds take the warp-wide minimum of (PM', l 2^S + k).
        constexpr int DEPTH = E >= 2 ? 2 : 1;
        Mask taken = 0;
        float c1 = 0.f, c2 = 0.f;
        int e1 = 0, e2 = 0;
        int avail = 0;
        // (x, ex) ranks before (y, ey): larger |value|, then smaller index
        auto better = [](float x, int ex, float y, int ey) {
            return fabsf(x) > fabsf(y) || (fabsf(x) == fabsf(y) && ex < ey);
        };
        if constexpr (E == 1) {
            c1 = v[0];
            avail = 1;
        } else if constexpr (E == 2) {
            const bool gg = fabsf(v[1]) > fabsf(v[0]);
            c1 = gg ? v[1] : v[0];
            e1 = gg ? 1 : 0;
            c2 = gg ? v[0] : v[1];
            e2 = gg ? 0 : 1;
            avail = 2;
        } else {
            // two independent scans (even and odd e) shorten the dependency chain; each keeps
            // its two best in (|c| descending, e ascending) order, then the lists merge
            float a1[2], a2[2];
            int i1[2], i2[2];
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const bool gg = fabsf(v[h + 2]) > fabsf(v[h]);
                a1[h] = gg ? v[h + 2] : v[h];
                i1[h] = gg ? h + 2 : h;
                a2[h] = gg ? v[h] : v[h + 2];
                i2[h] = gg ? h : h + 2;
            }
#pragma unroll
            for (int e = 4; e < E; e++) {
                const int h = e & 1;
                const float a = v[e];
                const bool g1 = fabsf(a) > fabsf(a1[h]);
                const bool g2 = fabsf(a) > fabsf(a2[h]);
                a2[h] = g1 ? a1[h] : (g2 ? a : a2[h]);
                i2[h] = g1 ? i1[h] : (g2 ? e : i2[h]);
                a1[h] = g1 ? a : a1[h];
                i1[h] = g1 ? e : i1[h];
            }
            const bool f0 = better(a1[0], i1[0], a1[1], i1[1]);
            c1 = f0 ? a1[0] : a1[1];
            e1 = f0 ? i1[0] : i1[1];
            const float sa = f0 ? a2[0] : a1[0];
            const int sai = f0 ? i2[0] : i1[0];
            const float sb = f0 ? a1[1] : a2[1];
            const int sbi = f0 ? i1[1] : i2[1];
            const bool f1 = better(sa, sai, sb, sbi);
            c2 = f1 ? sa : sb;
            e2 = f1 ? sai : sbi;
            avail = 2;
        }
        int used = 0;
        int my_par = 0, my_k = 0, my_neg = 0;
        float my_pm = 0.f;
#pragma unroll 1
        for (int q = 0; q < L; q++) {
            const float cc = used == 0 ? c1 : c2;
            const int ce = used == 0 ? e1 : e2;
            const float cpm = (act && used < avail) ? pml + 0.5f * (A - fabsf(cc)) : __int_as_float(0x7f800000);
            const unsigned cid = ((unsigned)((l << S) | (g + G * ce)) << 1) | (cc < 0.f ? 1u : 0u);
            // warp minimum of (PM', l 2^S + k): two single-instruction reductions on an
            // order-preserving integer image of PM', then on the index among the tied lanes
            const unsigned key = ordered_bits(cpm);
            const unsigned kmin = __reduce_min_sync(kFull, key);
            const unsigned imin = __reduce_min_sync(kFull, key == kmin ? cid : 0xffffffffu);
            const int cidx = (int)(imin >> 1);
            if (w.lane == q) {
                my_pm = ordered_float(kmin);
                my_par = cidx >> S;
                my_k = cidx & ((1 << S) - 1);
                my_neg = (int)(imin & 1u);
            }
            // the owner recognises itself: its key and index are the minimum
            if (key == kmin && cid == imin) {
                taken |= Mask(1) << ce;
                used++;
                if constexpr (E > DEPTH) {
                    if (used == DEPTH && q + 1 < L) {
                        // rare: both cached candidates were taken; rescan the untaken ones
                        bool h1 = false, h2 = false;
                        auto visit = [&](int e, float a) {
                            const bool ok = !((taken >> e) & 1);
                            const bool g1 = ok && (!h1 || fabsf(a) > fabsf(c1));
                            const bool g2 = ok && !g1 && (!h2 || fabsf(a) > fabsf(c2));
                            c2 = g1 ? c1 : (g2 ? a : c2);
                            e2 = g1 ? e1 : (g2 ? e : e2);
                            h2 = h2 || g2 || (g1 && h1);
                            c1 = g1 ? a : c1;
                            e1 = g1 ? e : e1;
                            h1 = h1 || g1;
                        };
                        if constexpr (M >= 9 && L <= 4) {
                            // a rolled loop over the lane's spectrum parked in its own slots of
                            // the leaf's shared-memory buffer (read only at the start of the
                            // leaf): 16% less code for the m = 9 trees, whose code exceeds the
                            // instruction caches, and no local memory; with L = 8 rescans are
                            // frequent enough, and smaller trees fit the caches, so the
                            // unrolled form below is faster there
                            float* mine = w.alpha + C::lvl_off(S) + l * ST + g;
#pragma unroll
                            for (int e = 0; e < E; e++) mine[G * e] = v[e];
#pragma unroll 1
                            for (int e = 0; e < E; e++) visit(e, mine[G * e]);
                        } else {
#pragma unroll
                            for (int e = 0; e < E; e++) visit(e, v[e]);
                        }
                        avail = (h1 ? 1 : 0) + (h2 ? 1 : 0);
                        used = 0;
                    }
                }
            }
        }
        fht_finish<S, OFF, PEND>(w, ps, my_par, my_k, my_neg, my_pm);
    }

    // The list step of an FHTL node and its decided bits: lane q < L holds the q-th survivor,
    // descended from path my_par with candidate (my_k, my_neg) and metric my_pm.
    template <int S, int OFF, unsigned PEND>
    __device__ __forceinline__ static void fht_finish(Warp& w, PState<M>& ps, int my_par, int my_k, int my_neg,
                                                      float my_pm) {
        reselect<OFF, PEND>(w, ps, my_par, my_pm);
        // decided bits x_j = <k, j> xor sign over the span
        constexpr int NB = 1 << S;
        if constexpr (NB >= 32) {
            constexpr int WPP = NB / 32;
            constexpr int TOT = L * WPP;
#pragma unroll
            for (int it = 0; it < (TOT + 31) / 32; it++) {
                const int idx = w.lane + 32 * it;
                const int q = idx < TOT ? idx / WPP : 0;
                const int kq = __shfl_sync(kFull, my_k, q);
                const int nq = __shfl_sync(kFull, my_neg, q);
                if (idx < TOT) {
                    const int wd = idx % WPP;
                    unsigned pat = 0;
#pragma unroll
                    for (int t = 0; t < 5; t++) {
                        const unsigned mt = t == 0 ? 0xAAAAAAAAu : t == 1 ? 0xCCCCCCCCu : t == 2 ? 0xF0F0F0F0u
                                           : t == 3 ? 0xFF00FF00u : 0xFFFF0000u;
                        if ((kq >> t) & 1) pat ^= mt;
                    }
                    if ((__popc((kq >> 5) & wd) & 1) ^ nq) pat = ~pat;
                    bitbuf(w, w.bsel, q)[OFF / 32 + wd] = pat;
                }
            }
            __syncwarp();
        } else {
            unsigned pat = 0;
#pragma unroll
            for (int j = 0; j < NB; j++) pat |= (unsigned)((__popc(my_k & j) & 1) ^ my_neg) << j;
            put_small_bits<OFF, NB>(w, pat);
        }
    }

    // ------------------------------------------------------------- SPCL leaf ---
    // RM(S-1, S) node (Eqs. (2)-(6)): parity, PM += p |alpha_lrb|, then tau = min(L, 2^S - 1)
    // list splits on the next least reliable positions (flip cost |alpha_i| + (1-2p)|alpha_lrb|,
    // each a 2L -> L selection by (PM, 2l + flip)), finally the least reliable bit restores
    // even parity.
    template <int S, int OFF, unsigned PEND>
    __device__ static void spc_leaf(Warp& w, PState<M>& ps) {
        if constexpr (LOCK) __syncthreads();  // see fht_leaf
        constexpr int NS = 1 << S;
        static_assert(NS <= 32, "SPC node larger than a warp word");
        constexpr int TAU = cmin(L, NS - 1);
        constexpr int ST = C::stride(S);
        const float* buf = w.alpha + C::lvl_off(S);
        // reliability order of every path's positions: (|alpha|, position) ascending
#pragma unroll
        for (int it = 0; it < (L * NS + 31) / 32; it++) {
            const int idx = w.lane + 32 * it;
            if (idx < L * NS) {
                const int l = idx / NS, i = idx % NS;
                const float* a = buf + l * ST;
                const float ai = fabsf(a[i]);
                int rank = 0;
#pragma unroll
                for (int j = 0; j < NS; j++) {
                    const float aj = fabsf(a[j]);
                    rank += (aj < ai) || (aj == ai && j < i);
                }
                w.spc[l * 32 + rank] = (uint8_t)i;
            }
        }
        __syncwarp();
        // Lane l < L keeps, for path l as SPC-entry ancestor, its LRB and, in split order, the
        // next TAU positions and reliabilities; every round takes the values of each path's
        // ancestor with shuffles, and the lanes then shift their own lists by one.
        const int me = w.lane < L ? w.lane : 0;
        const float* am = buf + me * ST;
        const int o0 = w.spc[me * 32];
        const float lrb = fabsf(am[o0]);
        float rel[TAU];
        int pos[TAU];
#pragma unroll
        for (int t = 0; t < TAU; t++) {
            pos[t] = w.spc[me * 32 + 1 + t];
            rel[t] = fabsf(am[pos[t]]);
        }
        float pm;
        int p;
        {
            unsigned hd0 = 0;
#pragma unroll
            for (int i = 0; i < NS; i++) hd0 |= (am[i] < 0.f ? 1u : 0u) << i;
            p = __popc(hd0) & 1;
            pm = ps.pm + (p ? lrb : 0.f);  // Eq. (3)
        }
        __syncwarp();  // the order lists are read; w.spc now holds the selection of each round
        uint8_t* sel = w.spc;
        unsigned flip = 0;
        int orig = me;
#pragma unroll 1
        for (int t = 1; t <= TAU; t++) {
            // the split position and the LRB belong to the path's SPC-entry ancestor `orig`
            const float r_o = __shfl_sync(kFull, rel[0], orig);
            const int itp = __shfl_sync(kFull, pos[0], orig);
            const float lrb_o = __shfl_sync(kFull, lrb, orig);
            const float pflip = pm + r_o + (p ? -lrb_o : lrb_o);  // Eq. (4)
            // candidate c = 2l + flip; every group of 2L lanes holds all candidates and
            // compares them against its share of the 2L, and the partial counts are summed
            constexpr int NC = 2 * L;
            if constexpr (NC > 32) {
                // 2L = 64 candidates (L = 32): lane t ranks candidates t and t + 32
                const int ca = w.lane, cb = w.lane + 32;
                const float ka = __shfl_sync(kFull, pm, ca >> 1), fa = __shfl_sync(kFull, pflip, ca >> 1);
                const float kb = __shfl_sync(kFull, pm, cb >> 1), fb = __shfl_sync(kFull, pflip, cb >> 1);
                const float pa = (ca & 1) ? fa : ka, pb = (cb & 1) ? fb : kb;
                int ra = 0, rb = 0;
#pragma unroll 4
                for (int c2 = 0; c2 < NC; c2++) {
                    const float o = __shfl_sync(kFull, c2 < 32 ? pa : pb, c2 & 31);
                    ra += (o < pa) || (o == pa && c2 < ca);
                    rb += (o < pb) || (o == pb && c2 < cb);
                }
                if (ra < L) sel[ra] = (uint8_t)ca;
                if (rb < L) sel[rb] = (uint8_t)cb;
            } else {
                constexpr int GRP = cmin(32 / NC, NC);  // lane groups sharing the comparisons
                constexpr int Q = NC / GRP;             // comparisons per group
                const int c = w.lane & (NC - 1);
                const int grp = (w.lane / NC) % GRP;
                const float kpm = __shfl_sync(kFull, pm, c >> 1);
                const float fpm = __shfl_sync(kFull, pflip, c >> 1);
                const float cpm = (c & 1) ? fpm : kpm;
                // rank of candidate c among the 2L by (PM, 2l + flip)
                int rank = 0;
#pragma unroll
                for (int k = 0; k < Q; k++) {
                    const int c2 = grp * Q + k;
                    const float o = __shfl_sync(kFull, cpm, c2);
                    rank += (o < cpm) || (o == cpm && c2 < c);
                }
#pragma unroll
                for (int d = NC; d < NC * GRP; d <<= 1) rank += __shfl_xor_sync(kFull, rank, d);
                // candidate of rank q goes to path q
                if (w.lane < 2 * L && rank < L) sel[rank] = (uint8_t)w.lane;
            }
            __syncwarp();
            const int mysrc = sel[me];
            __syncwarp();
            const int sp = mysrc >> 1;
            const bool fl = mysrc & 1;
            // state of the source path: metric, ancestor, flips, parity, split position
            const float n_kpm = __shfl_sync(kFull, pm, sp);
            const float n_fpm = __shfl_sync(kFull, pflip, sp);
            const float n_pm = fl ? n_fpm : n_kpm;
            const unsigned packed = __shfl_sync(kFull, (unsigned)orig | ((unsigned)p << 8) | ((unsigned)itp << 16), sp);
            const unsigned n_flip = __shfl_sync(kFull, flip, sp);
            pm = n_pm;
            orig = (int)(packed & 0xffu);
            const int n_it = (int)(packed >> 16);
            flip = fl ? (n_flip ^ (1u << n_it)) : n_flip;  // Eq. (5)
            p = fl ? (int)(((packed >> 8) & 1u) ^ 1u) : (int)((packed >> 8) & 1u);
#pragma unroll
            for (int k = 0; k + 1 < TAU; k++) {
                rel[k] = rel[k + 1];
                pos[k] = pos[k + 1];
            }
        }
        unsigned x;
        {
            const float* ao = buf + orig * ST;
            unsigned hd = 0;
#pragma unroll
            for (int i = 0; i < NS; i++) hd |= (ao[i] < 0.f ? 1u : 0u) << i;
            const int lo0 = __shfl_sync(kFull, o0, orig);
            x = (hd ^ flip) & ~(1u << lo0);
            x |= (unsigned)(__popc(x) & 1) << lo0;  // Eq. (6)
        }
        reselect<OFF, PEND>(w, ps, orig, pm);
        put_small_bits<OFF, NS>(w, x);
    }

    // --------------------------------------------------- permutation selection ---
    // 2L candidates: candidate c permutes the LLRs of source path c mod L; its reliability
    // LM_c = sum_{i < N_v/2} |f(tmp_i, tmp_{i+N_v/2})| (Algorithm 2, scoring of the candidates). For an
    // affine permutation, {pi(i), pi(i + N_v/2)} = {j, j ^ a} with a the image of the top
    // index bit, so LM_c = sum over the pairs {j, j ^ a} of min(|alpha_j|, |alpha_{j^a}|),
    // summed here with one representative j per pair (bit msb(a) clear). Returns, in lane
    // q < L, the candidate of rank q under (LM descending, c ascending).
    template <int S, typename Src>
    __device__ static int select_perms(Warp& w, const uint16_t* recs, Src src) {
        constexpr int C2 = 2 * L;
        constexpr int HALF = 1 << (S - 1);
        if constexpr (C2 > 32) {
            // 2L = 64 candidates (L = 32): lane t keeps LM of candidates t and t + 32, ranks
            // both, and the candidate of rank q is published to lane q through shared memory
            float lm0 = 0.f, lm1 = 0.f;
#pragma unroll 2
            for (int c = 0; c < C2; c++) {
                const uint16_t* r = recs + c * kRec;
                const int a = r[S - 1];
                const int h = 31 - __clz(a);
                const int lorg = c & (L - 1);
                float acc = 0.f;
#pragma unroll
                for (int t = 0; t < (HALF + 31) / 32; t++) {
                    const int jp = w.lane + 32 * t;
                    if (jp < HALF) {
                        const int j = insert_zero(jp, h);
                        acc += fminf(fabsf(src(lorg, j)), fabsf(src(lorg, j ^ a)));
                    }
                }
                acc = warp_sum(acc);
                if (w.lane == (c & 31)) {
                    if (c < 32) lm0 = acc;
                    else lm1 = acc;
                }
            }
            const int c0 = w.lane, c1 = w.lane + 32;
            int r0 = 0, r1 = 0;
#pragma unroll 4
            for (int c2 = 0; c2 < C2; c2++) {
                const float o = __shfl_sync(kFull, c2 < 32 ? lm0 : lm1, c2 & 31);
                r0 += (o > lm0) || (o == lm0 && c2 < c0);
                r1 += (o > lm1) || (o == lm1 && c2 < c1);
            }
            uint8_t* sel = w.spc;  // free outside SPC leaves
            __syncwarp();
            if (r0 < L) sel[r0] = (uint8_t)c0;
            if (r1 < L) sel[r1] = (uint8_t)c1;
            __syncwarp();
            const int mine = sel[w.lane];
            __syncwarp();
            return mine;
        }
        float mylm = 0.f;  // lane c keeps LM_c
        if constexpr (M >= 9 && !(M == 9 && L == 8)) {
            // candidates two at a time, each with a warp sum (the m = 9 trees exceed the
            // instruction caches: the fully unrolled form below measured 2-3.5% slower for
            // RM(2,9) with L = 4, but 3% faster for RM(3,9) with L = 8; longer lists and
            // longer codes spill in it)
#pragma unroll 2
            for (int c = 0; c < C2; c++) {
                const uint16_t* r = recs + c * kRec;
                const int a = r[S - 1];
                const int h = 31 - __clz(a);
                const int lorg = c & (L - 1);
                float acc = 0.f;
#pragma unroll
                for (int t = 0; t < (HALF + 31) / 32; t++) {
                    const int jp = w.lane + 32 * t;
                    if (jp < HALF) {
                        const int j = insert_zero(jp, h);
                        acc += fminf(fabsf(src(lorg, j)), fabsf(src(lorg, j ^ a)));
                    }
                }
                acc = warp_sum(acc);
                if (w.lane == c) mylm = acc;
            }
        } else {
            // smaller trees: every lane's partial LM of every candidate ...
            constexpr int LG = cilog2(C2);
            float part[C2];
#pragma unroll
            for (int c = 0; c < C2; c++) {
                const uint16_t* r = recs + c * kRec;
                const int a = r[S - 1];
                const int h = 31 - __clz(a);
                const int lorg = c & (L - 1);
                float acc = 0.f;
#pragma unroll
                for (int t = 0; t < (HALF + 31) / 32; t++) {
                    const int jp = w.lane + 32 * t;
                    if (jp < HALF) {
                        const int j = insert_zero(jp, h);
                        acc += fminf(fabsf(src(lorg, j)), fabsf(src(lorg, j ^ a)));
                    }
                }
                part[c] = acc;
            }
            // ... reduced and scattered over the butterfly d = 16, 8, ..., 1: the first LG stages
            // halve the candidates a lane holds (it keeps one half and adds the partner's copy of
            // it), the rest add across lanes holding the same candidate. Every addition is the one
            // a warp sum of that candidate's partials makes, so the totals are bitwise equal to it.
#pragma unroll
            for (int st = 0; st < 5; st++) {
                const int d = 16 >> st;
                if (st < LG) {
                    const int n = C2 >> st;  // candidates held before this stage
                    const bool up = (w.lane & d) != 0;
#pragma unroll
                    for (int k = 0; k < C2 / 2; k++) {
                        if (k < n / 2) {
                            const float keep = up ? part[k + n / 2] : part[k];
                            const float give = up ? part[k] : part[k + n / 2];
                            part[k] = keep + __shfl_xor_sync(kFull, give, d);
                        }
                    }
                } else {
                    part[0] += __shfl_xor_sync(kFull, part[0], d);
                }
            }
            // lanes with (lane >> (5 - LG)) == c hold LM_c; lane c < C2 takes it
            mylm = __shfl_sync(kFull, part[0], (w.lane & (C2 - 1)) << (5 - LG));
        }
        // rank of candidate `lane` by (LM descending, c ascending); lane q < L takes rank q
        int rank = 0;
#pragma unroll
        for (int c2 = 0; c2 < C2; c2++) {
            const float o = __shfl_sync(kFull, mylm, c2);
            rank += (o > mylm) || (o == mylm && c2 < w.lane);
        }
        int mine = 0;
#pragma unroll
        for (int q = 0; q < L; q++) {
            const unsigned b = __ballot_sync(kFull, w.lane < C2 && rank == q);
            if (w.lane == q) mine = __ffs(b) - 1;
        }
        return mine;
    }

    // ------------------------------------------------------------- tree walk ---
    template <int RR, int S, int OFF, bool ROOT, bool SPINE, unsigned PEND>
    __device__ static void node(Warp& w, PState<M>& ps) {
        if constexpr (RR == 1) {
            fht_leaf<S, OFF, PEND>(w, ps);
        } else if constexpr (RR == S - 1) {
            spc_leaf<S, OFF, PEND>(w, ps);
        } else {
            constexpr bool PERM = SPINE;  // 1 < RR < S - 1 holds here
            constexpr int H = 1 << (S - 1);
            constexpr int STC = C::stride(S - 1);
            float* child = w.alpha + C::lvl_off(S - 1);
            constexpr int LEVEL = M - S;  // permuted-level index on the spine
            const uint16_t* lrec = w.rec + LEVEL * 2 * L * kRec;
            // LLRs of this node for path l at position j
            // a deeper permuted node keeps its permuted copy in the level's second buffer
            // (LEAN: in the level's own buffer, the unpermuted LLRs staged below)
            constexpr bool ALT = PERM && !ROOT && !C::LEAN;
            const float* nodebuf = w.alpha + (ALT ? C::alt_off(S) : C::lvl_off(S));
            constexpr int STN = C::stride(S);
            if constexpr (ROOT) {
                // every path's LLRs are y, so candidate c's permuted LLRs are y through the
                // composed permutation pi^init_{c mod L} o pi_c (one GA(m) element)
                const int c = select_perms<S>(w, lrec, [&](int, int j) { return w.y[j]; });
                ps.rootc = c;
                ps.pm = __shfl_sync(kFull, ps.pm, c & (L - 1));  // the source path's start metric
            } else if constexpr (PERM) {
                const float* src = w.alpha + C::lvl_off(S);
                const int c = select_perms<S>(w, lrec, [&](int l, int j) { return src[l * STN + j]; });
                // path q takes source path c mod L through pi_c
                const float npm = __shfl_sync(kFull, ps.pm, (w.lane < L ? c : 0) & (L - 1));
                reselect<OFF, PEND>(w, ps, c % L, npm);
                ps.selc[S] = c;
                const float* from = src;
                if constexpr (C::LEAN) {
                    // stage the L unpermuted paths in the lower levels' buffers (offset 0, free
                    // until the first descent below this level; lvl_off(S) >= L * STN floats)
                    float* stage = w.alpha;
#pragma unroll 4
                    for (int i = w.lane; i < L * STN; i += 32) stage[i] = src[i];
                    __syncwarp();
                    from = stage;
                }
                float* dst = w.alpha + (C::LEAN ? C::lvl_off(S) : C::alt_off(S));
#pragma unroll 1
                for (int q = 0; q < L; q++) {
                    const int cq = __shfl_sync(kFull, c, q);
                    const uint16_t* r = lrec + cq * kRec;
                    const float* s_src = from + (cq % L) * STN;
                    const int base = ga_lane_base(r, S, w.lane);
#pragma unroll
                    for (int t = 0; t < ((1 << S) + 31) / 32; t++) {
                        const int i = w.lane + 32 * t;
                        if (i < (1 << S)) dst[q * STN + i] = s_src[base ^ ga_hi(r, S, t)];
                    }
                }
                __syncwarp();
            }
            // this node's LLRs were just written with path l in slot l
            if (w.lane < L) ps.slot[S] = w.lane;
            // f: left child RM(RR-1, S-1) (Algorithm 2)
            if constexpr (ROOT) {
#pragma unroll 1
                for (int l = 0; l < L; l++) {
                    const int cl = __shfl_sync(kFull, ps.rootc, l);
                    const uint16_t* r = lrec + cl * kRec;
                    const int a = r[S - 1];
                    const int base = ga_lane_base(r, S - 1, w.lane);
#pragma unroll
                    for (int t = 0; t < (H + 31) / 32; t++) {
                        const int i = w.lane + 32 * t;
                        if (i < H) {
                            const int j = base ^ ga_hi(r, S - 1, t);
                            child[l * STC + i] = fminsum(w.y[j], w.y[j ^ a]);
                        }
                    }
                }
            } else if constexpr (H >= 32) {
#pragma unroll 4  // independent paths: 4 chains in flight
                for (int l = 0; l < L; l++)
#pragma unroll
                    for (int t = 0; t < H / 32; t++) {
                        const int i = w.lane + 32 * t;
                        child[l * STC + i] = fminsum(nodebuf[l * STN + i], nodebuf[l * STN + i + H]);
                    }
            } else {
#pragma unroll
                for (int it = 0; it < (L * H + 31) / 32; it++) {
                    const int idx = w.lane + 32 * it;
                    if (idx < L * H) {
                        const int l = idx / H, i = idx % H;
                        child[l * STC + i] = fminsum(nodebuf[l * STN + i], nodebuf[l * STN + i + H]);
                    }
                }
            }
            __syncwarp();
            node<RR - 1, S - 1, OFF, false, SPINE, (PEND | (1u << S))>(w, ps);
            // g: right child RM(RR, S-1) from the path's own ancestor LLRs (Algorithm 2)
            if constexpr (ROOT) {
#pragma unroll 1
                for (int l = 0; l < L; l++) {
                    const int cl = __shfl_sync(kFull, ps.rootc, l);
                    const uint16_t* r = lrec + cl * kRec;
                    const int a = r[S - 1];
                    const int base = ga_lane_base(r, S - 1, w.lane);
                    const uint32_t* bl = bitbuf(w, w.bsel, l);
#pragma unroll
                    for (int t = 0; t < (H + 31) / 32; t++) {
                        const int i = w.lane + 32 * t;
                        if (i < H) {
                            const int j = base ^ ga_hi(r, S - 1, t);
                            const unsigned xb = (bl[(OFF + i) >> 5] >> ((OFF + i) & 31)) & 1u;
                            child[l * STC + i] = g_fn(w.y[j], w.y[j ^ a], xb);
                        }
                    }
                }
            } else if constexpr (H >= 32) {
                static_assert(OFF % 32 == 0, "spans of 64 or more bits are word aligned");
#pragma unroll 4
                for (int l = 0; l < L; l++) {
                    const int sl = __shfl_sync(kFull, ps.slot[S], l);
                    const uint32_t* bl = bitbuf(w, w.bsel, l) + OFF / 32;
                    const float* src = nodebuf + sl * STN;
#pragma unroll
                    for (int t = 0; t < H / 32; t++) {
                        const int i = w.lane + 32 * t;
                        child[l * STC + i] = g_fn(src[i], src[i + H], (bl[t] >> w.lane) & 1u);
                    }
                }
            } else {
#pragma unroll
                for (int it = 0; it < (L * H + 31) / 32; it++) {
                    const int idx = w.lane + 32 * it;
                    const int l = idx < L * H ? idx / H : 0;
                    const int sl = __shfl_sync(kFull, ps.slot[S], l);
                    if (idx < L * H) {
                        const int i = idx % H;
                        const uint32_t* bl = bitbuf(w, w.bsel, l);
                        const unsigned xb = (bl[(OFF + i) >> 5] >> ((OFF + i) & 31)) & 1u;
                        child[l * STC + i] = g_fn(nodebuf[sl * STN + i], nodebuf[sl * STN + i + H], xb);
                    }
                }
            }
            __syncwarp();
            node<RR, S - 1, OFF + H, false, false, PEND>(w, ps);
            // combine x_v = (x_gamma ^ x_lambda, x_gamma) (Algorithm 2); the root does this for
            // the winning path only
            if constexpr (!ROOT) {
                if constexpr (H >= 32) {
                    constexpr int WH = H / 32;
#pragma unroll
                    for (int it = 0; it < (L * WH + 31) / 32; it++) {
                        const int idx = w.lane + 32 * it;
                        if (idx < L * WH) {
                            uint32_t* b = bitbuf(w, w.bsel, idx / WH);
                            const int wd = idx % WH;
                            b[OFF / 32 + wd] ^= b[(OFF + H) / 32 + wd];
                        }
                    }
                } else {
                    if (w.lane < L) {
                        uint32_t* wd = bitbuf(w, w.bsel, w.lane) + OFF / 32;
                        const unsigned mh = (1u << H) - 1u;
                        *wd ^= ((*wd >> ((OFF % 32) + H)) & mh) << (OFF % 32);
                    }
                }
                __syncwarp();
                if constexpr (PERM) {
                    // undo pi*_l on the node's span (Algorithm 2): x[pi(i)] = x'[i]
                    static_assert(OFF == 0, "permuted nodes lie on the left spine");
                    constexpr int SB = 1 << S;
                    if constexpr (SB >= 32) {
                        constexpr int SW = SB / 32;
                        // gather form x[j] = x'[pi^-1(j)]: word t of the result is the
                        // ballot of lane j's source bits; lane t keeps it until every lane
                        // has read the path's old bits
                        static_assert(SW <= 32, "one result word per lane");
#pragma unroll 1
                        for (int l = 0; l < L; l++) {
                            const int cl = __shfl_sync(kFull, ps.selc[S], l);
                            const uint16_t* ri = w.rec_inv + (LEVEL * 2 * L + cl) * kRec;
                            uint32_t* b = bitbuf(w, w.bsel, l);
                            const int base = ga_lane_base(ri, S, w.lane);
                            unsigned mine = 0;
#pragma unroll
                            for (int t = 0; t < SW; t++) {
                                const int srcp = base ^ ga_hi(ri, S, t);
                                const unsigned word = __ballot_sync(kFull, (b[srcp >> 5] >> (srcp & 31)) & 1u);
                                if (w.lane == t) mine = word;
                            }
                            __syncwarp();
                            if (w.lane < SW) b[w.lane] = mine;
                            __syncwarp();
                        }
                    } else {
                        if (w.lane < L) {
                            const uint16_t* r = lrec + ps.selc[S] * kRec;
                            uint32_t* b = bitbuf(w, w.bsel, w.lane);
                            const unsigned old = b[0];
                            unsigned nw = 0;
#pragma unroll
                            for (int i = 0; i < SB; i++)
                                if ((old >> i) & 1u) nw |= 1u << ga_apply(r, S, i);
                            const unsigned mask = (1u << SB) - 1u;
                            b[0] = (old & ~mask) | nw;
                        }
                        __syncwarp();
                    }
                }
            }
        }
    }

    // Runs one decoder (Algorithm 2 from the root); returns the best path's metric and its
    // root permutation. The path's bits stay in its bit buffer (see emit()).
    __device__ static float run(Warp& w, int& c0) {
        PState<M> ps;
        ps.pm = (w.single && w.lane != 0) ? __int_as_float(0x7f800000) : 0.f;
        ps.rootc = 0;
#pragma unroll
        for (int s = 0; s <= M; s++) {
            ps.slot[s] = w.lane < L ? w.lane : 0;
            ps.selc[s] = 0;
        }
        w.bsel = 0;
        node<R, M, 0, true, true, 0u>(w, ps);
        // the list is sorted by metric: path 0 is the decoder's best (Algorithm 5)
        c0 = __shfl_sync(kFull, ps.rootc, 0);
        return __shfl_sync(kFull, ps.pm, 0);
    }

    // Root combine and un-permutation of path 0 into `dst` (the codeword in the channel
    // domain): x_root = (x_gamma ^ x_lambda, x_gamma), then x[sigma(i)] = x'[i] with
    // sigma = pi^init o pi* the path's composed root permutation (Algorithm 2),
    // read through the inverse map the host stores after the decoder's records.
    __device__ static void emit(Warp& w, int c0, uint32_t* dst) {
        uint32_t* b = bitbuf(w, w.bsel, 0);
        constexpr int H = N / 2;
        if constexpr (H >= 32) {
            for (int wd = w.lane; wd < H / 32; wd += 32) b[wd] ^= b[H / 32 + wd];
        } else if (w.lane == 0) {
            b[0] ^= (b[0] >> H) & ((1u << H) - 1u);
        }
        __syncwarp();
        // gather form x[j] = x'[sigma^-1(j)]: word t of the codeword is the ballot of lane j's
        // source bits
        static_assert(NW <= 32, "one codeword word per lane");
        const uint16_t* ri = w.rec_inv + c0 * kRec;
        const int base = ga_lane_base(ri, M, w.lane);
        unsigned mine = 0;
#pragma unroll
        for (int t = 0; t < NW; t++) {
            const int srcp = base ^ ga_hi(ri, M, t);
            const bool in = w.lane + 32 * t < N;
            const unsigned word = __ballot_sync(kFull, in && ((b[srcp >> 5] >> (srcp & 31)) & 1u));
            if (w.lane == t) mine = word;
        }
        if (w.lane < NW) dst[w.lane] = mine;
        __syncwarp();
    }
};

// Block shared memory, common to every configuration: the frame LLRs first (at offset 0 of
// the block's shared memory, so that the permutation gathers address them with the index
// alone: measured +6% on RM(2,9) and +11% on RM(3,9) against placing them after the tables),
// per-warp (metric, decoder) reduction slots, the decoders' permutation records (SMEM_NREC per
// decoder) and the K information positions, then one area of warp_stride bytes per warp.
__host__ __device__ constexpr int frame_fixed_bytes(int rec_elems, int K, int N, int W) {
    return ((N * 4 + W * 8 + 15) / 16) * 16 + ((rec_elems * 2 + K * 2 + 15) / 16) * 16;
}

template <int M, int R, int L>
__host__ constexpr int Cfg<M, R, L>::fixed_bytes(int P, int K, int W) {
    return frame_fixed_bytes(P * SMEM_NREC * kRec, K, N, W);
}

// The forward maps of P decoders (per decoder `per` elements, followed in the device table by
// as many of inverse maps) into shared memory, whole block.
__device__ __forceinline__ void copy_maps(uint16_t* dst, const uint16_t* recs, int P, int per) {
    for (int i = threadIdx.x; i < P * per; i += blockDim.x) dst[i] = recs[(i / per) * 2 * per + i % per];
}

struct FrameSmem {
    float* y;         // frame LLRs (N of the largest code the block decodes)
    float* redpm;     // per warp: best metric of the frame so far
    int* redp;        // per warp: its decoder
    uint16_t* rec;    // records of the decoders (SMEM_NREC per decoder)
    uint16_t* info;   // their information positions
    uint8_t* wbase;   // the warp areas
    int warp_stride;  // bytes per warp area
};

// The layout of frame_fixed_bytes for codes of up to N positions and W warps.
__device__ __forceinline__ FrameSmem carve_smem(uint8_t* smem, int rec_elems, int K, int warp_stride, int N, int W) {
    FrameSmem s;
    s.y = reinterpret_cast<float*>(smem);
    s.redpm = s.y + N;
    s.redp = reinterpret_cast<int*>(s.redpm + W);
    const int tables = ((N * 4 + W * 8 + 15) / 16) * 16;
    s.rec = reinterpret_cast<uint16_t*>(smem + tables);
    s.info = s.rec + rec_elems;
    s.wbase = smem + tables + ((rec_elems * 2 + K * 2 + 15) / 16) * 16;
    s.warp_stride = warp_stride;
    return s;
}

// What the decode of one frame reads and writes (output pointers may be null except info_out).
struct FrameJob {
    const uint16_t* recs;  // the decoders' device tables (maps, then inverse maps, per decoder)
    const void* llr;     // [frames][N] of dtype
    int dtype;
    float qclamp;        // |code| clamp for I16 inputs
    int P, K;
    int single;          // one live initial path (FHT-FSCL without permutations)
    uint32_t* info_out;  // [frames][ceil(K/32)]
    uint32_t* cw_out;    // [frames][ceil(N/32)]
    float* pm_out;       // [frames]
    int32_t* best_out;   // [frames]
};

// Decodes frame f of a job with the whole block (Algorithm 5 over the P decoders, split
// round-robin over the warps). The block's records (unless LEAN) and information positions
// must already be in shared memory; the first barrier also publishes them. LOCK: see Decoder.
template <int M, int R, int L, bool LOCK, bool TC = false>
__device__ __forceinline__ void decode_frame(const FrameJob& j, const FrameSmem& sm, int64_t f) {
    using C = Cfg<M, R, L>;
    using D = Decoder<M, R, L, LOCK, TC>;
    constexpr int N = C::N;
    constexpr int NW = C::NW;
    const int W = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    float* s_y = sm.y;
    float* s_redpm = sm.redpm;
    int* s_redp = sm.redp;
    uint8_t* wbase = sm.wbase;
    uint8_t* mine = wbase + warp * sm.warp_stride;
    Warp w;
    w.alpha = reinterpret_cast<float*>(mine);
    w.bits = reinterpret_cast<uint32_t*>(mine + C::OFF_BITS);
    w.xtmp = reinterpret_cast<uint32_t*>(mine + C::OFF_XTMP);
    w.best = reinterpret_cast<uint32_t*>(mine + C::OFF_BEST);
    w.spc = mine + C::OFF_SPC;
    w.y = s_y;
    w.lane = lane;
    w.single = j.single != 0;

    __syncthreads();
    // frame LLRs into shared memory, widened to float
    if (j.dtype == IN_F32) {
        const float4* src = reinterpret_cast<const float4*>(static_cast<const float*>(j.llr) + f * N);
        for (int i = threadIdx.x; i < N / 4; i += blockDim.x) reinterpret_cast<float4*>(s_y)[i] = src[i];
    } else if (j.dtype == IN_I8) {
        // 16 codes per 16-byte load (N >= 16, frames 16-byte aligned)
        const uint4* src = reinterpret_cast<const uint4*>(static_cast<const int8_t*>(j.llr) + f * N);
        for (int i = threadIdx.x; i < N / 16; i += blockDim.x) {
            const uint4 q = src[i];
            const uint32_t wv[4] = {q.x, q.y, q.z, q.w};
            float4* dst = reinterpret_cast<float4*>(s_y) + 4 * i;
#pragma unroll
            for (int c = 0; c < 4; c++)  // byte b of the word, sign-extended
                dst[c] = make_float4((float)((int32_t)(wv[c] << 24) >> 24), (float)((int32_t)(wv[c] << 16) >> 24),
                                     (float)((int32_t)(wv[c] << 8) >> 24), (float)((int32_t)wv[c] >> 24));
        }
    } else if (j.dtype == IN_F16) {
        // 8 halves per 16-byte load
        const uint4* src = reinterpret_cast<const uint4*>(static_cast<const __half*>(j.llr) + f * N);
        for (int i = threadIdx.x; i < N / 8; i += blockDim.x) {
            const uint4 q = src[i];
            const uint32_t wv[4] = {q.x, q.y, q.z, q.w};
            float2* dst = reinterpret_cast<float2*>(s_y) + 4 * i;
#pragma unroll
            for (int c = 0; c < 4; c++) dst[c] = __half22float2(*reinterpret_cast<const __half2*>(&wv[c]));
        }
    } else {
        // 8 codes per 16-byte load, clamped so that every sum stays exact in FP32
        const uint4* src = reinterpret_cast<const uint4*>(static_cast<const int16_t*>(j.llr) + f * N);
        for (int i = threadIdx.x; i < N / 8; i += blockDim.x) {
            const uint4 q = src[i];
            const uint32_t wv[4] = {q.x, q.y, q.z, q.w};
            float2* dst = reinterpret_cast<float2*>(s_y) + 4 * i;
#pragma unroll
            for (int c = 0; c < 4; c++)
                dst[c] = make_float2(fminf(fmaxf((float)((int32_t)(wv[c] << 16) >> 16), -j.qclamp), j.qclamp),
                                     fminf(fmaxf((float)((int32_t)wv[c] >> 16), -j.qclamp), j.qclamp));
        }
    }
    __syncthreads();
    float best = __int_as_float(0x7f800000);
    int bestp = -1;
    // rounds of W decoders, one per warp, with a block barrier after every round. With LOCK
    // every warp runs a decoder in every round (the leaves hold block barriers): when W does
    // not divide P, a warp without a decoder of its own in the last round repeats decoder
    // P - 1 and discards the result.
    for (int p0 = 0; p0 < j.P; p0 += W) {
        const int p = p0 + warp;
        if (LOCK || p < j.P) {
            const int pr = p < j.P ? p : j.P - 1;
            w.rec = C::LEAN ? j.recs + 2 * pr * C::NREC * kRec : sm.rec + pr * C::NREC * kRec;
            w.rec_inv = j.recs + (2 * pr + 1) * C::NREC * kRec;
            int c0;
            const float pm = D::run(w, c0);
            if (p < j.P && (bestp < 0 || pm < best)) {  // strict: earlier decoders win ties (Algorithm 5)
                best = pm;
                bestp = p;
                D::emit(w, c0, w.best);
            }
        }
        __syncthreads();
    }
    if (lane == 0) {
        s_redpm[warp] = best;
        s_redp[warp] = bestp;
    }
    __syncthreads();
    if (warp == 0) {
        // the winner over warps by (metric, decoder index)
        float bp = __int_as_float(0x7f800000);
        int bw = 0, bpp = 1 << 30;
        for (int q = 0; q < W; q++) {
            const float v = s_redpm[q] == s_redpm[q] ? s_redpm[q] : __int_as_float(0x7f800000);  // NaN: last
            const int pq = s_redp[q];
            if (pq >= 0 && (v < bp || (v == bp && pq < bpp))) {
                bp = v;
                bpp = pq;
                bw = q;
            }
        }
        uint32_t* cw = reinterpret_cast<uint32_t*>(wbase + bw * sm.warp_stride + C::OFF_BEST);
        if (j.cw_out)
            for (int wd = lane; wd < NW; wd += 32) j.cw_out[f * NW + wd] = cw[wd];
        if (lane == 0) {
            if (j.pm_out) j.pm_out[f] = bp;
            if (j.best_out) j.best_out[f] = bpp;
        }
        // u = x G^{(x)m}: u_i = XOR of x_j over j containing i
        uint32_t* u = w.xtmp;
        for (int wd = lane; wd < NW; wd += 32) {
            unsigned v = cw[wd];
            if (M > 0) v ^= (v >> 1) & 0x55555555u;
            if (M > 1) v ^= (v >> 2) & 0x33333333u;
            if (M > 2) v ^= (v >> 4) & 0x0F0F0F0Fu;
            if (M > 3) v ^= (v >> 8) & 0x00FF00FFu;
            if (M > 4) v ^= (v >> 16) & 0x0000FFFFu;
            u[wd] = v;
        }
        __syncwarp();
#pragma unroll
        for (int t = 5; t < M; t++) {
            const int d = 1 << (t - 5);
            for (int wd = lane; wd < NW; wd += 32)
                if (!(wd & d)) u[wd] ^= u[wd | d];
            __syncwarp();
        }
        const int KW = (j.K + 31) / 32;
        for (int it = 0; it < KW; it++) {
            const int jj = lane + 32 * it;
            unsigned bit = 0;
            if (jj < j.K) {
                const int pos = sm.info[jj];
                bit = (u[pos >> 5] >> (pos & 31)) & 1u;
            }
            const unsigned word = __ballot_sync(kFull, bit);
            if (lane == 0) j.info_out[f * KW + it] = word;
        }
    }
}

template <int M, int R, int L, bool TC = false>
__global__ void __launch_bounds__(32 * kMaxWarps, 1) pfht_kernel(LaunchArgs args) {
    using C = Cfg<M, R, L>;
    extern __shared__ __align__(16) uint8_t smem[];
    const int rec_elems = args.P * C::SMEM_NREC * kRec;
    const FrameSmem sm = carve_smem(smem, rec_elems, args.K, C::WARP_BYTES, C::N, blockDim.x >> 5);
    copy_maps(sm.rec, args.recs, args.P, C::SMEM_NREC * kRec);
    for (int i = threadIdx.x; i < args.K; i += blockDim.x) sm.info[i] = args.info[i];
    FrameJob j;
    j.recs = args.recs;
    j.llr = args.llr;
    j.dtype = args.dtype;
    j.qclamp = args.qclamp;
    j.P = args.P;
    j.K = args.K;
    j.single = args.single_start;
    j.info_out = args.info_out;
    j.cw_out = args.cw_out;
    j.pm_out = args.pm_out;
    j.best_out = args.best_out;
    for (int64_t f = blockIdx.x; f < args.n_frames; f += gridDim.x) decode_frame<M, R, L, true, TC>(j, sm, f);
}

}  // namespace rmdec_dev
