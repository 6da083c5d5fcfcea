// Decoders of RM(1, m) and RM(m-1, m): codes whose root is itself an FHTL or SPCL node.
//
// Algorithm 2 reaches such a root before any path extension in the permutation domain, and
// undoes the initial permutations only in the branch of permuted nodes; the initial
// permutations are automorphisms of the code, which would only copy the same candidate words
// into every path. Each decoder therefore decodes y directly with one live path, and the best
// path of the list is the maximum-likelihood word:
//   RM(1, m): the Walsh-Hadamard spectrum c of y (Algorithm 4); the word of index k with the
//     largest |c_k| (ties: smaller k) and sign [c_k < 0], path metric (sum|y| - |c_k|) / 2
//     (Eq. (8));
//   RM(m-1, m): the hard decision, with the least reliable position (ties: smaller index)
//     flipped when the parity is odd, path metric p |y_lrb| (Eqs. (2)-(3), (6)).
// All P decoders decide alike, so decoder 0 wins (Algorithm 5, strict comparison).
//
// One warp per frame; position i of the frame sits in lane i % 32, register i / 32.
#include <cstdint>

#include <cuda_fp16.h>

#include "pfht_kernel.cuh"
#include "rmdec_internal.h"

namespace rmdec_dev {

template <int M, bool SPC>
__global__ void __launch_bounds__(256) mlroot_kernel(LaunchArgs a) {
    constexpr int N = 1 << M;
    constexpr int E = N >= 32 ? N / 32 : 1;  // positions per lane
    constexpr int NW = (N + 31) / 32;        // codeword words
    const int lane = threadIdx.x & 31;
    const int W = blockDim.x >> 5;
    const int KW = (a.K + 31) / 32;
    const unsigned inf_bits = 0x7f800000u;
    for (int64_t f = (int64_t)blockIdx.x * W + (threadIdx.x >> 5); f < a.n_frames; f += (int64_t)gridDim.x * W) {
        float v[E];
#pragma unroll
        for (int e = 0; e < E; e++) {
            const int i = lane + 32 * e;
            float x = 0.f;
            if (i < N) {
                const int64_t o = f * N + i;
                if (a.dtype == IN_F32) x = static_cast<const float*>(a.llr)[o];
                else if (a.dtype == IN_I8) x = (float)static_cast<const int8_t*>(a.llr)[o];
                else if (a.dtype == IN_F16) x = __half2float(static_cast<const __half*>(a.llr)[o]);
                else x = fminf(fmaxf((float)static_cast<const int16_t*>(a.llr)[o], -a.qclamp), a.qclamp);
            }
            v[e] = x;
        }
        uint32_t cw = 0;  // lane w < NW holds codeword word w
        float pm;
        if constexpr (!SPC) {
            float A = 0.f;
#pragma unroll
            for (int e = 0; e < E; e++) A += fabsf(v[e]);
#pragma unroll
            for (int d = 16; d >= 1; d >>= 1) A += __shfl_xor_sync(kFull, A, d);
            // butterflies (u, w) -> (u + w, u - w): register bits of the index, then lane bits
#pragma unroll
            for (int h = 1; h < E; h <<= 1)
#pragma unroll
                for (int e = 0; e < E; e++)
                    if (!(e & h)) {
                        const float p = v[e], q = v[e + h];
                        v[e] = p + q;
                        v[e + h] = p - q;
                    }
#pragma unroll
            for (int d = 1; d < (N < 32 ? N : 32); d <<= 1) {
#pragma unroll
                for (int e = 0; e < E; e++) {
                    const float o = __shfl_xor_sync(kFull, v[e], d);
                    v[e] = (lane & d) ? o - v[e] : v[e] + o;
                }
            }
            // largest |c_k|, ties to the smaller k (within a lane k grows with e)
            float best = fabsf(v[0]);
            float cb = v[0];
            int be = 0;
#pragma unroll
            for (int e = 1; e < E; e++)
                if (fabsf(v[e]) > best) {
                    best = fabsf(v[e]);
                    cb = v[e];
                    be = e;
                }
            const bool valid = lane < N;
            const unsigned key = valid ? __float_as_uint(best) : 0u;  // |c| >= 0: bits order as values
            const unsigned kmax = __reduce_max_sync(kFull, key);
            const unsigned kidx = __reduce_min_sync(kFull, (valid && key == kmax) ? (unsigned)(lane + 32 * be) : 0xffffffffu);
            const float cbest = __shfl_sync(kFull, cb, kidx & 31);
            const int k = (int)kidx;
            const unsigned neg = cbest < 0.f ? 1u : 0u;
            pm = 0.5f * (A - __uint_as_float(kmax));
            // codeword x_j = <k, j> xor neg, word w = bits 32 w .. 32 w + 31
            if (lane < NW) {
                unsigned pat = 0;
#pragma unroll
                for (int t = 0; t < 5; t++) {
                    const unsigned mt = t == 0 ? 0xAAAAAAAAu : t == 1 ? 0xCCCCCCCCu : t == 2 ? 0xF0F0F0F0u
                                       : t == 3 ? 0xFF00FF00u : 0xFFFF0000u;
                    if ((k >> t) & 1) pat ^= mt;
                }
                if ((__popc((unsigned)(k >> 5) & (unsigned)lane) & 1) ^ neg) pat = ~pat;
                cw = N >= 32 ? pat : (pat & ((1u << N) - 1u));
            }
        } else {
            // hard decisions, parity and the least reliable position (ties: smaller index)
            int par = 0;
#pragma unroll
            for (int e = 0; e < E; e++) {
                const unsigned b = __ballot_sync(kFull, lane + 32 * e < N && v[e] < 0.f);
                par ^= __popc(b) & 1;
                if (lane == e) cw = b;
            }
            float lo = fabsf(v[0]);
            int le = 0;
#pragma unroll
            for (int e = 1; e < E; e++)
                if (fabsf(v[e]) < lo) {
                    lo = fabsf(v[e]);
                    le = e;
                }
            const bool valid = lane < N;
            const unsigned key = valid ? __float_as_uint(lo) : inf_bits;
            const unsigned kmin = __reduce_min_sync(kFull, key);
            const unsigned lrb = __reduce_min_sync(kFull, (valid && key == kmin) ? (unsigned)(lane + 32 * le) : 0xffffffffu);
            pm = par ? __uint_as_float(kmin) : 0.f;
            if (par && lane == (int)(lrb >> 5)) cw ^= 1u << (lrb & 31);
        }
        if (a.cw_out && lane < NW) a.cw_out[f * NW + lane] = cw;
        if (lane == 0) {
            if (a.pm_out) a.pm_out[f] = pm;
            if (a.best_out) a.best_out[f] = 0;
        }
        // u = x G^{(x)m}: u_i = XOR of x_j over j containing i (within words, then across)
        uint32_t u = cw;
        if (M > 0) u ^= (u >> 1) & 0x55555555u;
        if (M > 1) u ^= (u >> 2) & 0x33333333u;
        if (M > 2) u ^= (u >> 4) & 0x0F0F0F0Fu;
        if (M > 3) u ^= (u >> 8) & 0x00FF00FFu;
        if (M > 4) u ^= (u >> 16) & 0x0000FFFFu;
#pragma unroll
        for (int t = 5; t < M; t++) {
            const int d = 1 << (t - 5);
            const uint32_t o = __shfl_xor_sync(kFull, u, d);
            if (!(lane & d)) u ^= o;
        }
        for (int it = 0; it < KW; it++) {
            const int jj = lane + 32 * it;
            const int pos = jj < a.K ? (int)a.info[jj] : 0;
            const uint32_t wd = __shfl_sync(kFull, u, pos >> 5);
            const unsigned word = __ballot_sync(kFull, jj < a.K && ((wd >> (pos & 31)) & 1u));
            if (lane == 0) a.info_out[f * KW + it] = word;
        }
    }
}

}  // namespace rmdec_dev

namespace rmdec_host {

namespace {
template <int M, bool SPC>
void mlroot_entry(KernelEntry* e) {
    e->fn = reinterpret_cast<const void*>(&rmdec_dev::mlroot_kernel<M, SPC>);
    e->warp_bytes = 0;
    e->nrec = 0;
    e->fixed_bytes = [](int, int, int) { return 0; };
}
template <int M>
bool mlroot_case(int r, KernelEntry* e) {
    if (r == 1) {
        mlroot_entry<M, false>(e);
        return true;
    }
    if (r == M - 1) {
        mlroot_entry<M, true>(e);
        return true;
    }
    return false;
}
}  // namespace

bool lookup_mlroot(int m, int r, KernelEntry* e) {
    switch (m) {
        case 2: return mlroot_case<2>(r, e);
        case 3: return mlroot_case<3>(r, e);
        case 4: return mlroot_case<4>(r, e);
        case 5: return mlroot_case<5>(r, e);
        case 6: return mlroot_case<6>(r, e);
        case 7: return mlroot_case<7>(r, e);
        case 8: return mlroot_case<8>(r, e);
        case 9: return mlroot_case<9>(r, e);
        case 10: return mlroot_case<10>(r, e);
    }
    return false;
}

}  // namespace rmdec_host
