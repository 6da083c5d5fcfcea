// Aut-SSC-P baseline decoder for RM(r, m): SSC decoding (repetition nodes RM(0, s), single
// parity-check nodes RM(s-1, s), min-sum f and g elsewhere, Section II-B) of P_ssc copies of
// the frame permuted by GA(m) elements, keeping the candidate with the smallest correlation
// discrepancy sum_i |y_i| [x_i != HD(y_i)] (earliest permutation on ties). This is the
// permuted SSC decoder the paper compares against (Section III-B, Table 5, Fig. 6).
//
// A CTA owns one frame at a time; its warps split the permutations; one warp runs one SSC
// pass with all LLRs of the pass in shared memory (one buffer per tree level).
#include <cstdint>

#include "pfht_kernel.cuh"
#include "rmdec_internal.h"

namespace rmdec_dev {

template <int M, int R>
struct SscCfg {
    static constexpr int N = 1 << M;
    static constexpr int NW = N >= 32 ? N / 32 : 1;
    static __host__ __device__ constexpr int lvl_off(int s) {
        int o = 0;
        for (int t = 1; t < s; t++) o += 1 << t;
        return o;
    }
    static constexpr int ALPHA_FLOATS = lvl_off(M);
    // warp area: alpha | bits (NW) | xtmp (NW) | best (NW)
    static constexpr int OFF_BITS = ALPHA_FLOATS * 4;
    static constexpr int OFF_XTMP = OFF_BITS + NW * 4;
    static constexpr int OFF_BEST = OFF_XTMP + NW * 4;
    static constexpr int WARP_BYTES = (OFF_BEST + NW * 4 + 15) / 16 * 16;
    static __host__ constexpr int fixed_bytes(int P, int K, int W) {
        return ((N * 4 + W * 8 + 15) / 16) * 16 + ((P * kRec * 2 + K * 2 + 15) / 16) * 16;
    }
};

template <int M, int R>
struct Ssc {
    using C = SscCfg<M, R>;
    static constexpr int N = C::N;

    template <int OFF, int NB>
    __device__ static void put_bits(uint32_t* bits, int lane, unsigned v) {
        if constexpr (NB >= 32) {
            for (int wd = lane; wd < NB / 32; wd += 32) bits[OFF / 32 + wd] = v;
        } else {
            if (lane == 0) {
                const unsigned mask = ((1u << NB) - 1u) << (OFF % 32);
                bits[OFF / 32] = (bits[OFF / 32] & ~mask) | ((v << (OFF % 32)) & mask);
            }
        }
        __syncwarp();
    }

    // LLRs of node (S, ROOT): the root reads y through the permutation r.
    template <int RR, int S, int OFF, bool ROOT>
    __device__ static void node(float* alpha, uint32_t* bits, const float* y, const uint16_t* r, int lane) {
        constexpr int NS = 1 << S;
        const float* a = alpha + C::lvl_off(S);
        if constexpr (RR == 0) {
            // repetition node: all bits = sign of the LLR sum
            float acc = 0.f;
            for (int i = lane; i < NS; i += 32) acc += a[i];
            acc = warp_sum(acc);
            put_bits<OFF, NS>(bits, lane, acc < 0.f ? 0xffffffffu : 0u);
        } else if constexpr (RR == S - 1) {
            // single parity check (Wagner): hard decisions, flip the least reliable on odd parity
            static_assert(NS <= 32, "SPC node fits a warp");
            const float v = lane < NS ? a[lane] : 0.f;
            const unsigned hd = __ballot_sync(kFull, lane < NS && v < 0.f);
            float best = lane < NS ? fabsf(v) : __int_as_float(0x7f800000);
            int bi = lane;
#pragma unroll
            for (int d = 16; d >= 1; d >>= 1) {
                const float ob = __shfl_xor_sync(kFull, best, d);
                const int oi = __shfl_xor_sync(kFull, bi, d);
                const bool take = ob < best || (ob == best && oi < bi);
                best = take ? ob : best;
                bi = take ? oi : bi;
            }
            const unsigned x = hd ^ ((unsigned)(__popc(hd) & 1) << bi);
            put_bits<OFF, NS>(bits, lane, x);
        } else {
            constexpr int H = NS / 2;
            float* child = alpha + C::lvl_off(S - 1);
            const int amask = ROOT ? r[S - 1] : 0;
            const int base = ROOT ? ga_lane_base(r, S - 1, lane) : 0;
#pragma unroll
            for (int t = 0; t < (H + 31) / 32; t++) {
                const int i = lane + 32 * t;
                if (i < H) {
                    float u, v;
                    if constexpr (ROOT) {
                        const int j = base ^ ga_hi(r, S - 1, t);
                        u = y[j];
                        v = y[j ^ amask];
                    } else {
                        u = a[i];
                        v = a[i + H];
                    }
                    child[i] = fminsum(u, v);
                }
            }
            __syncwarp();
            node<RR - 1, S - 1, OFF, false>(alpha, bits, y, r, lane);
#pragma unroll
            for (int t = 0; t < (H + 31) / 32; t++) {
                const int i = lane + 32 * t;
                if (i < H) {
                    float u, v;
                    if constexpr (ROOT) {
                        const int j = base ^ ga_hi(r, S - 1, t);
                        u = y[j];
                        v = y[j ^ amask];
                    } else {
                        u = a[i];
                        v = a[i + H];
                    }
                    const int xb = (bits[(OFF + i) >> 5] >> ((OFF + i) & 31)) & 1;
                    child[i] = xb ? v - u : v + u;
                }
            }
            __syncwarp();
            node<RR, S - 1, OFF + H, false>(alpha, bits, y, r, lane);
            if constexpr (H >= 32) {
                for (int wd = lane; wd < H / 32; wd += 32) bits[OFF / 32 + wd] ^= bits[(OFF + H) / 32 + wd];
            } else {
                if (lane == 0) {
                    uint32_t* wd = bits + OFF / 32;
                    *wd ^= ((*wd >> ((OFF % 32) + H)) & ((1u << H) - 1u)) << (OFF % 32);
                }
            }
            __syncwarp();
        }
    }
};

template <int M, int R>
__global__ void __launch_bounds__(256) autssc_kernel(LaunchArgs args) {
    using C = SscCfg<M, R>;
    constexpr int N = C::N;
    constexpr int NW = C::NW;
    extern __shared__ __align__(16) uint8_t smem[];
    const int W = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int P = args.P;
    const int K = args.K;
    // the frame LLRs at offset 0 (the permutation gathers then address them by index alone),
    // reduction slots, permutation records, information positions, warp areas
    float* s_y = reinterpret_cast<float*>(smem);
    float* s_red = s_y + N;
    int* s_redq = reinterpret_cast<int*>(s_red + W);
    const int tables = ((N * 4 + W * 8 + 15) / 16) * 16;
    uint16_t* s_rec = reinterpret_cast<uint16_t*>(smem + tables);
    uint16_t* s_info = s_rec + P * kRec;
    uint8_t* wbase = smem + tables + ((P * kRec * 2 + K * 2 + 15) / 16) * 16;
    uint8_t* mine = wbase + warp * C::WARP_BYTES;
    float* alpha = reinterpret_cast<float*>(mine);
    uint32_t* bits = reinterpret_cast<uint32_t*>(mine + C::OFF_BITS);
    uint32_t* xtmp = reinterpret_cast<uint32_t*>(mine + C::OFF_XTMP);
    uint32_t* bestcw = reinterpret_cast<uint32_t*>(mine + C::OFF_BEST);

    for (int i = threadIdx.x; i < P * kRec; i += blockDim.x) s_rec[i] = args.recs[i];
    for (int i = threadIdx.x; i < K; i += blockDim.x) s_info[i] = args.info[i];

    for (int64_t f = blockIdx.x; f < args.n_frames; f += gridDim.x) {
        __syncthreads();
        if (args.dtype == IN_F32) {
            const float4* src = reinterpret_cast<const float4*>(static_cast<const float*>(args.llr) + f * N);
            for (int i = threadIdx.x; i < N / 4; i += blockDim.x) reinterpret_cast<float4*>(s_y)[i] = src[i];
        } else if (args.dtype == IN_I8) {
            const int8_t* src = static_cast<const int8_t*>(args.llr) + f * N;
            for (int i = threadIdx.x; i < N; i += blockDim.x) s_y[i] = (float)src[i];
        } else if (args.dtype == IN_F16) {
            const __half* src = static_cast<const __half*>(args.llr) + f * N;
            for (int i = threadIdx.x; i < N; i += blockDim.x) s_y[i] = __half2float(src[i]);
        } else {
            const int16_t* src = static_cast<const int16_t*>(args.llr) + f * N;
            for (int i = threadIdx.x; i < N; i += blockDim.x)
                s_y[i] = fminf(fmaxf((float)src[i], -args.qclamp), args.qclamp);
        }
        __syncthreads();
        float best = __int_as_float(0x7f800000);
        int bestq = -1;
        for (int q = warp; q < P; q += W) {
            const uint16_t* r = s_rec + q * kRec;
            Ssc<M, R>::template node<R, M, 0, true>(alpha, bits, s_y, r, lane);
            // discrepancy of the candidate, evaluated in the permuted domain (it is invariant)
            const int base = ga_lane_base(r, M, lane);
            float d = 0.f;
#pragma unroll
            for (int t = 0; t < (N + 31) / 32; t++) {
                const int i = lane + 32 * t;
                if (i < N) {
                    const float v = s_y[base ^ ga_hi(r, M, t)];
                    const int xb = (bits[i >> 5] >> (i & 31)) & 1;
                    if (xb != (v < 0.f ? 1 : 0)) d += fabsf(v);
                }
            }
            d = warp_sum(d);
            if (bestq < 0 || d < best) {
                best = d;
                bestq = q;
                for (int wd = lane; wd < NW; wd += 32) xtmp[wd] = 0;
                __syncwarp();
#pragma unroll
                for (int t = 0; t < (N + 31) / 32; t++) {
                    const int i = lane + 32 * t;
                    if (i < N && ((bits[i >> 5] >> (i & 31)) & 1)) {
                        const int dstp = base ^ ga_hi(r, M, t);
                        atomicOr(&xtmp[dstp >> 5], 1u << (dstp & 31));
                    }
                }
                __syncwarp();
                for (int wd = lane; wd < NW; wd += 32) bestcw[wd] = xtmp[wd];
            }
            __syncwarp();
        }
        if (lane == 0) {
            s_red[warp] = best;
            s_redq[warp] = bestq;
        }
        __syncthreads();
        if (warp == 0) {
            float bd = __int_as_float(0x7f800000);
            int bw = 0, bq = 1 << 30;
            for (int q = 0; q < W; q++) {
                const float v = s_red[q] == s_red[q] ? s_red[q] : __int_as_float(0x7f800000);  // NaN: last
                if (s_redq[q] >= 0 && (v < bd || (v == bd && s_redq[q] < bq))) {
                    bd = v;
                    bq = s_redq[q];
                    bw = q;
                }
            }
            const uint32_t* cw = reinterpret_cast<const uint32_t*>(wbase + bw * C::WARP_BYTES + C::OFF_BEST);
            if (args.cw_out)
                for (int wd = lane; wd < NW; wd += 32) args.cw_out[f * NW + wd] = cw[wd];
            if (lane == 0) {
                if (args.pm_out) args.pm_out[f] = bd;
                if (args.best_out) args.best_out[f] = bq;
            }
            uint32_t* u = xtmp;
            for (int wd = lane; wd < NW; wd += 32) {
                unsigned v = cw[wd];
                v ^= (v >> 1) & 0x55555555u;
                v ^= (v >> 2) & 0x33333333u;
                v ^= (v >> 4) & 0x0F0F0F0Fu;
                v ^= (v >> 8) & 0x00FF00FFu;
                v ^= (v >> 16) & 0x0000FFFFu;
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
            const int KW = (K + 31) / 32;
            for (int it = 0; it < KW; it++) {
                const int j = lane + 32 * it;
                unsigned bit = 0;
                if (j < K) {
                    const int pos = s_info[j];
                    bit = (u[pos >> 5] >> (pos & 31)) & 1u;
                }
                const unsigned word = __ballot_sync(kFull, bit);
                if (lane == 0) args.info_out[f * KW + it] = word;
            }
        }
    }
}

}  // namespace rmdec_dev

namespace rmdec_host {

#define RMDEC_SSC_ENTRY(M, R)                                                        \
    if (m == M && r == R) {                                                          \
        e->fn = reinterpret_cast<const void*>(&rmdec_dev::autssc_kernel<M, R>);      \
        e->warp_bytes = rmdec_dev::SscCfg<M, R>::WARP_BYTES;                         \
        e->nrec = 1;                                                                 \
        e->fixed_bytes = [](int P, int K, int W) { return rmdec_dev::SscCfg<M, R>::fixed_bytes(P, K, W); }; \
        return true;                                                                 \
    }

bool lookup_autssc(int m, int r, KernelEntry* e) {
    RMDEC_SSC_ENTRY(4, 1) RMDEC_SSC_ENTRY(4, 2)
    RMDEC_SSC_ENTRY(5, 1) RMDEC_SSC_ENTRY(5, 2) RMDEC_SSC_ENTRY(5, 3)
    RMDEC_SSC_ENTRY(6, 1) RMDEC_SSC_ENTRY(6, 2) RMDEC_SSC_ENTRY(6, 3)
    RMDEC_SSC_ENTRY(7, 1) RMDEC_SSC_ENTRY(7, 2) RMDEC_SSC_ENTRY(7, 3)
    RMDEC_SSC_ENTRY(8, 1) RMDEC_SSC_ENTRY(8, 2) RMDEC_SSC_ENTRY(8, 3)
    RMDEC_SSC_ENTRY(9, 1) RMDEC_SSC_ENTRY(9, 2) RMDEC_SSC_ENTRY(9, 3)
    return false;
}

}  // namespace rmdec_host
