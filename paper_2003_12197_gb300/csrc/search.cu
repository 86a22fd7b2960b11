// Encrypted search kernels of the HERS library (Alg 7 server loop; Eq. 4;
// the ciphertext multiply of Alg 5 with its rounding and relinearisation
// moved after the sum over the d dimensions):
//
//   tensor   X_k = sum_i tensor_k(probe_i, gallery_i^b), k = 0, 1, 2, exactly,
//            as residues mod q1 q2 p1 p2 p3 in the NTT domain (pointwise);
//   intt     X_k back to the coefficient domain (15 polynomials per block);
//   scale    c_k = [round(t X_k / q)]_q, exact (RNS, no floating point);
//   keyswitch (c0, c1, c2) -> (c0 + sum_j D_j evk_j0, c1 + sum_j D_j evk_j1),
//            D_j = c2 mod q_j, once per gallery block.
#include "common.cuh"
#include "internal.h"

namespace hers {

// ---------------------------------------------------------------- tensor accumulate
//
// Thread (k, l) of CTA (tile, l, group) owns coefficient k of limb l for NB
// consecutive gallery blocks.  Operands are split-stored (a = ah 2^27 + al,
// 27-bit halves), so every partial product is one 32x32 -> 64-bit
// multiply-add on the integer pipe, accumulated without reduction:
//   T0 = sum a0 b0,  T1 = sum (a0 b1 + a1 b0),  T2 = sum a1 b1
// each kept as (lo, mid, hi) with value lo + mid 2^27 + hi 2^54.  A
// partial product is < 2^54 and mid of T1 takes 4 per dimension, so 128
// dimensions fit in 64 bits; longer sums are folded mod p every 128.
constexpr int TENSOR_THREADS = 256;
constexpr int TENSOR_CHUNK = 128;

template <int NB>
__global__ void __launch_bounds__(TENSOR_THREADS) k_tensor(const uint64_t* __restrict__ gal,
                                                           const uint64_t* __restrict__ probe,
                                                           uint64_t* __restrict__ acc,
                                                           uint64_t nblocks, uint32_t d) {
    const int k = blockIdx.x * TENSOR_THREADS + threadIdx.x;
    const int l = blockIdx.y;
    const uint64_t b0 = (uint64_t)blockIdx.z * NB;
    const uint64_t p = c_mod[l];
    const size_t poly = (size_t)5 * N;  // stride between the two polys of a ct
    const size_t ct = 2 * poly;         // stride between cts

    int nb = (int)((nblocks - b0) < (uint64_t)NB ? (nblocks - b0) : NB);
    uint64_t fold[NB][3];
#pragma unroll
    for (int j = 0; j < NB; j++) fold[j][0] = fold[j][1] = fold[j][2] = 0;

    const uint64_t* pa = probe + (size_t)l * N + k;
    const uint64_t* ga = gal + (b0 * d) * ct + (size_t)l * N + k;
    const size_t gstride = (size_t)d * ct;  // between consecutive gallery blocks

    for (uint32_t i0 = 0; i0 < d; i0 += TENSOR_CHUNK) {
        const uint32_t i1 = min(d, i0 + TENSOR_CHUNK);
        uint64_t s[NB][9];
#pragma unroll
        for (int j = 0; j < NB; j++)
#pragma unroll
            for (int r = 0; r < 9; r++) s[j][r] = 0;
#pragma unroll 2
        for (uint32_t i = i0; i < i1; i++) {
            const uint64_t A0 = __ldg(pa + (size_t)i * ct), A1 = __ldg(pa + (size_t)i * ct + poly);
            const uint32_t a0l = (uint32_t)A0, a0h = (uint32_t)(A0 >> 32);
            const uint32_t a1l = (uint32_t)A1, a1h = (uint32_t)(A1 >> 32);
#pragma unroll
            for (int j = 0; j < NB; j++) {
                if (j < nb) {
                    const uint64_t* g = ga + j * gstride + (size_t)i * ct;
                    const uint64_t B0 = __ldcs(g), B1 = __ldcs(g + poly);
                    const uint32_t b0l = (uint32_t)B0, b0h = (uint32_t)(B0 >> 32);
                    const uint32_t b1l = (uint32_t)B1, b1h = (uint32_t)(B1 >> 32);
                    s[j][0] += (uint64_t)a0l * b0l;
                    s[j][1] += (uint64_t)a0l * b0h + (uint64_t)a0h * b0l;
                    s[j][2] += (uint64_t)a0h * b0h;
                    s[j][3] += (uint64_t)a0l * b1l + (uint64_t)a1l * b0l;
                    s[j][4] += (uint64_t)a0l * b1h + (uint64_t)a0h * b1l + (uint64_t)a1l * b0h +
                               (uint64_t)a1h * b0l;
                    s[j][5] += (uint64_t)a0h * b1h + (uint64_t)a1h * b0h;
                    s[j][6] += (uint64_t)a1l * b1l;
                    s[j][7] += (uint64_t)a1l * b1h + (uint64_t)a1h * b1l;
                    s[j][8] += (uint64_t)a1h * b1h;
                }
            }
        }
        // fold: value = lo + mid 2^27 + hi 2^54 mod p
#pragma unroll
        for (int j = 0; j < NB; j++)
#pragma unroll
            for (int c = 0; c < 3; c++) {
                uint64_t v = shoup_lazy(s[j][3 * c + 0], 1, c_one_s[l], p) +
                             shoup_lazy(s[j][3 * c + 1], c_r27[l], c_r27_s[l], p) +
                             shoup_lazy(s[j][3 * c + 2], c_r54[l], c_r54_s[l], p) + fold[j][c];
                fold[j][c] = reduce64(v, l);  // v < 7p
            }
    }
#pragma unroll
    for (int j = 0; j < NB; j++)
        if (j < nb)
#pragma unroll
            for (int c = 0; c < 3; c++) acc[(((b0 + j) * 3 + c) * 5 + l) * N + k] = fold[j][c];
}

// ---------------------------------------------------------------- tensor accumulate, TMA pipeline
//
// Same result as k_tensor, organised for HBM streaming on sm_103a:
//  - CTA (tile, l, group): TT = 256 consumer threads, one coefficient each,
//    for NB gallery blocks, plus one producer warp;
//  - the producer's elected lane streams, per dimension i, the probe rows
//    (2 polys x TT words) and the NB gallery rows (NB x 2 polys x TT words) into
//    a STAGES-deep shared-memory ring with cp.async.bulk (2 KiB per row),
//    completion tracked by one "full" mbarrier per stage; consumers release a
//    stage through its "empty" mbarrier (one arrival per consumer warp);
//  - consumers use two-level Karatsuba on the 27-bit digits: with
//    x = xh 2^27 + xl,  x y = xh yh 2^54 + ((xh+xl)(yh+yl) - xh yh - xl yl) 2^27 + xl yl,
//    and T1 = (A0+A1)(B0+B1) - T0 - T2, so each (dimension, coefficient, limb,
//    block) costs 9 IMAD.WIDE.U32 instead of 16.  The largest partial product
//    is (2^29)^2 = 2^58, so sums are folded mod p every KCHUNK = 32 dimensions.
//  - a wait that exceeds WAIT_LIMIT polls sets *err and ends the thread's work.
constexpr int TT = 256;
constexpr int KCHUNK = 32;

template <int NB, int STAGES>
__global__ void __launch_bounds__(TT + 32) k_tensor_tma(const uint64_t* __restrict__ gal,
                                                        const uint64_t* __restrict__ probe,
                                                        uint64_t* __restrict__ acc,
                                                        uint64_t nblocks, uint32_t d, int* err) {
    extern __shared__ __align__(128) uint64_t sm[];
    __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES];
    constexpr int ROWS = 2 + 2 * NB;  // rows of TT words per stage
    const int tile = blockIdx.x, l = blockIdx.y;
    const uint64_t b0 = (uint64_t)blockIdx.z * NB;
    const int nb = (int)((nblocks - b0) < (uint64_t)NB ? (nblocks - b0) : NB);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t poly = (size_t)5 * N, ct = 2 * poly;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], TT / 32);
        }
        mbar_fence_init();
    }
    __syncthreads();

    if (warp == TT / 32) {  // producer warp
        if (lane == 0) {
            const uint64_t pol_g = policy_evict_first(), pol_p = policy_evict_last();
            const uint32_t bytes = (uint32_t)((2 + 2 * nb) * TT * 8);
            const uint64_t* pb = probe + (size_t)l * N + (size_t)tile * TT;
            const uint64_t* gb = gal + b0 * d * ct + (size_t)l * N + (size_t)tile * TT;
            uint32_t issued = 0;
            for (uint32_t i = 0; i < d; i++) {
                const int st = (int)(i % STAGES);
                if (i >= STAGES && !mbar_wait(&empty[st], ((i / STAGES) + 1) & 1)) {
                    atomicOr(err, 2);
                    break;
                }
                issued = i + 1;
                uint64_t* dst = sm + (size_t)st * ROWS * TT;
                mbar_expect_tx(&full[st], bytes);
                bulk_g2s(dst, pb + (size_t)i * ct, TT * 8, &full[st], pol_p);
                bulk_g2s(dst + TT, pb + (size_t)i * ct + poly, TT * 8, &full[st], pol_p);
                for (int j = 0; j < nb; j++) {
                    const uint64_t* g = gb + (size_t)j * d * ct + (size_t)i * ct;
                    bulk_g2s(dst + (2 + 2 * j) * TT, g, TT * 8, &full[st], pol_g);
                    bulk_g2s(dst + (3 + 2 * j) * TT, g + poly, TT * 8, &full[st], pol_g);
                }
            }
            // drain: the copies of the last stages issued have landed before this
            // thread leaves (bounded; consumers wait on the same phases)
            for (uint32_t i = issued > STAGES ? issued - STAGES : 0; i < issued; i++)
                if (!mbar_wait(&full[i % STAGES], (i / STAGES) & 1)) atomicOr(err, 2);
        }
        return;
    }

    // consumers
    const int t = threadIdx.x;
    const uint64_t p = c_mod[l];
    uint64_t fold[NB][3];
#pragma unroll
    for (int j = 0; j < NB; j++) fold[j][0] = fold[j][1] = fold[j][2] = 0;
    bool ok = true;
    for (uint32_t i0 = 0; i0 < d && ok; i0 += KCHUNK) {
        const uint32_t i1 = min(d, i0 + KCHUNK);
        uint64_t s[NB][9];  // per block: LL0 HH0 MM0 | LL2 HH2 MM2 | LLk HHk MMk
#pragma unroll
        for (int j = 0; j < NB; j++)
#pragma unroll
            for (int r = 0; r < 9; r++) s[j][r] = 0;
        for (uint32_t i = i0; i < i1; i++) {
            const int st = (int)(i % STAGES);
            if (!mbar_wait(&full[st], (i / STAGES) & 1)) {
                atomicOr(err, 2);
                ok = false;
                break;
            }
            const uint64_t* row = sm + (size_t)st * ROWS * TT + t;
            const uint64_t A0 = row[0], A1 = row[TT];
            const uint32_t a0l = (uint32_t)A0, a0h = (uint32_t)(A0 >> 32);
            const uint32_t a1l = (uint32_t)A1, a1h = (uint32_t)(A1 >> 32);
            const uint32_t a0s = a0l + a0h, a1s = a1l + a1h;
            const uint32_t sal = a0l + a1l, sah = a0h + a1h, sas = sal + sah;
#pragma unroll
            for (int j = 0; j < NB; j++) {
                if (j < nb) {
                    const uint64_t B0 = row[(2 + 2 * j) * TT], B1 = row[(3 + 2 * j) * TT];
                    const uint32_t b0l = (uint32_t)B0, b0h = (uint32_t)(B0 >> 32);
                    const uint32_t b1l = (uint32_t)B1, b1h = (uint32_t)(B1 >> 32);
                    const uint32_t b0s = b0l + b0h, b1s = b1l + b1h;
                    const uint32_t sbl = b0l + b1l, sbh = b0h + b1h, sbs = sbl + sbh;
                    s[j][0] += (uint64_t)a0l * b0l;
                    s[j][1] += (uint64_t)a0h * b0h;
                    s[j][2] += (uint64_t)a0s * b0s;
                    s[j][3] += (uint64_t)a1l * b1l;
                    s[j][4] += (uint64_t)a1h * b1h;
                    s[j][5] += (uint64_t)a1s * b1s;
                    s[j][6] += (uint64_t)sal * sbl;
                    s[j][7] += (uint64_t)sah * sbh;
                    s[j][8] += (uint64_t)sas * sbs;
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[st]);
        }
        // fold the chunk: value = LL + (MM - HH - LL) 2^27 + HH 2^54 (mod p)
#pragma unroll
        for (int j = 0; j < NB; j++) {
            uint64_t v[3];
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const uint64_t LL = s[j][3 * c], HH = s[j][3 * c + 1], MM = s[j][3 * c + 2];
                v[c] = reduce64(shoup_lazy(LL, 1, c_one_s[l], p) +
                                    shoup_lazy(MM - HH - LL, c_r27[l], c_r27_s[l], p) +
                                    shoup_lazy(HH, c_r54[l], c_r54_s[l], p),
                                l);
            }
            // T0 = v0, T2 = v1, T1 = K - T0 - T2 with K = v2
            fold[j][0] = add_mod(fold[j][0], v[0], p);
            fold[j][2] = add_mod(fold[j][2], v[1], p);
            fold[j][1] = add_mod(fold[j][1], sub_mod(sub_mod(v[2], v[0], p), v[1], p), p);
        }
    }
    if (!ok) return;
    const int k = tile * TT + t;
#pragma unroll
    for (int j = 0; j < NB; j++)
        if (j < nb)
#pragma unroll
            for (int c = 0; c < 3; c++) acc[(((b0 + j) * 3 + c) * 5 + l) * N + k] = fold[j][c];
}

// ---------------------------------------------------------------- batched NTTs
// CTA per polynomial of a contiguous [npolys][N] array; modulus index
// mod_off + (P % mod_period).
template <bool INV>
__global__ void __launch_bounds__(NTT_THREADS) k_ntt_batch(const uint64_t* __restrict__ tw,
                                                           uint64_t* __restrict__ data,
                                                           int mod_period, int mod_off) {
    extern __shared__ uint64_t sm[];
    const uint64_t P = blockIdx.x;
    const int mi = mod_off + (int)(P % (uint64_t)mod_period);
    uint64_t* g = data + P * N;
    for (int k = threadIdx.x; k < N; k += blockDim.x) sm[k] = g[k];
    if (INV) ntt_inv_mod(sm, tw, mi);
    else ntt_fwd_mod(sm, tw, mi);
    for (int k = threadIdx.x; k < N; k += blockDim.x) g[k] = sm[k];
}

// ---------------------------------------------------------------- exact scale-and-round
//
// Thread per (b, poly c, k).  X has residues x_0..x_4 mod (q1, q2, p1, p2, p3),
// |X| < q P / 2.  With r = [t X]_q centred, Y = (t X - r) / q is an integer
// and equals round(t X / q) (|r| < q/2, q odd: no tie), |Y| < 2^150 < P/2:
//   Y mod p_i = (t x_i - r) q^-1 mod p_i,   i = p1, p2, p3;
//   Y from its three residues by mixed radix (Garner), centred by comparing
//   the digits with those of (P-1)/2;   c = Y mod q_l, l = 1, 2.
// Writes c to C[b][c][l][N] and, for c = 2, the relinearisation digits
// D_1 = c2 mod q1, D_2 = c2 mod q2 reduced into both limbs:
// KS[b][0] = D_1 mod q1, [1] = D_1 mod q2, [2] = D_2 mod q1, [3] = D_2 mod q2.
__global__ void __launch_bounds__(256) k_scale_round(const uint64_t* __restrict__ X,
                                                     uint64_t* __restrict__ C,
                                                     uint64_t* __restrict__ KS) {
    const int k = blockIdx.x * 256 + threadIdx.x;
    const int c = blockIdx.y;
    const uint64_t b = blockIdx.z;
    const uint64_t* x = X + ((b * 3 + c) * 5) * N + k;
    const uint64_t x0 = x[0], x1 = x[N], x2 = x[2 * N], x3 = x[3 * N], x4 = x[4 * N];
    const uint64_t q1 = c_mod[0], q2 = c_mod[1];

    // r = [t X]_q
    const uint64_t a1 = shoup(x0, T_PLAIN, c_t_s[0], q1);
    const uint64_t a2 = shoup(x1, T_PLAIN, c_t_s[1], q2);
    const Lifted R = lift_q(a1, a2);
    uint64_t y[3];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const int mi = 2 + i;
        const uint64_t p = c_mod[mi];
        const uint64_t xi = i == 0 ? x2 : (i == 1 ? x3 : x4);
        const uint64_t rm = lifted_mod(R, mi, a2);
        const uint64_t tx = shoup(xi, T_PLAIN, c_t_s[mi], p);
        y[i] = shoup(sub_mod(tx, rm, p), c_qinv_p[i], c_qinv_p_s[i], p);
    }
    // mixed radix Y = y1 + p1 z2 + p1 p2 z3
    const uint64_t p2 = c_mod[3], p3 = c_mod[4];
    const uint64_t z1 = y[0];
    const uint64_t z2 = shoup(sub_mod(y[1], csub(z1, p2), p2), P1INV_P2, P1INV_P2_S, p2);
    uint64_t t3 = shoup(sub_mod(y[2], csub(z1, p3), p3), P1INV_P3, P1INV_P3_S, p3);
    const uint64_t z3 = shoup(sub_mod(t3, csub(z2, p3), p3), P2INV_P3, P2INV_P3_S, p3);
    const bool neg = (z3 > HALFP_D3) || (z3 == HALFP_D3 && (z2 > HALFP_D2 || (z2 == HALFP_D2 && z1 > HALFP_D1)));
    uint64_t out[2];
#pragma unroll
    for (int l = 0; l < 2; l++) {
        const uint64_t q = c_mod[l];
        uint64_t v = add_mod(z1, shoup(z2, c_p1_mod_q[l], c_p1_mod_q_s[l], q), q);
        v = add_mod(v, shoup(z3, c_p1p2_mod_q[l], c_p1p2_mod_q_s[l], q), q);
        if (neg) v = sub_mod(v, c_p_mod_q[l], q);
        out[l] = v;
        C[((b * 3 + c) * 2 + l) * N + k] = v;
    }
    if (c == 2) {
        uint64_t* ks = KS + b * 4 * N + k;
        ks[0] = out[0];
        ks[N] = csub(out[0], q2);
        ks[2 * N] = out[1];
        ks[3 * N] = out[1];
    }
}

// ---------------------------------------------------------------- key switch
// KS (NTT domain) x evk_j (NTT, Shoup): O[b][c][l] = sum_j D_j evk_j[c][l].
__global__ void __launch_bounds__(256) k_ks_mul(const uint64_t* __restrict__ KS,
                                                const uint64_t* __restrict__ evk_ntt,
                                                uint64_t* __restrict__ O) {
    const int k = blockIdx.x * 256 + threadIdx.x;
    const int l = blockIdx.y;
    const uint64_t b = blockIdx.z;
    const uint64_t q = c_mod[l];
    const uint64_t D1 = KS[(b * 4 + l) * N + k], D2 = KS[(b * 4 + 2 + l) * N + k];
#pragma unroll
    for (int c = 0; c < 2; c++) {
        const uint64_t* e1 = evk_ntt + (size_t)(((0 * 2 + c) * 2 + l) * 2) * N;
        const uint64_t* e2 = evk_ntt + (size_t)(((1 * 2 + c) * 2 + l) * 2) * N;
        const uint64_t v = shoup_lazy(D1, e1[k], e1[N + k], q) + shoup_lazy(D2, e2[k], e2[N + k], q);
        O[((b * 2 + c) * 2 + l) * N + k] = reduce64(v, l);
    }
}

// out[b][c][l] = C[b][c][l] + O[b][c][l] mod q_l (O in the coefficient domain)
__global__ void __launch_bounds__(256) k_ks_finish(const uint64_t* __restrict__ C,
                                                   const uint64_t* __restrict__ O,
                                                   uint64_t* __restrict__ out) {
    const int k = blockIdx.x * 256 + threadIdx.x;
    const int l = blockIdx.y & 1, c = blockIdx.y >> 1;
    const uint64_t b = blockIdx.z;
    const uint64_t q = c_mod[l];
    out[((b * 2 + c) * 2 + l) * N + k] =
        add_mod(C[((b * 3 + c) * 2 + l) * N + k], O[((b * 2 + c) * 2 + l) * N + k], q);
}

// ---------------------------------------------------------------- pipeline
// Workspace per block: X [3][5][N] (reused for O [2][2][N]), C [3][2][N], KS [4][N].
cudaError_t launch_search(const uint64_t* tw, const DevKeys& k, const uint64_t* gallery,
                          uint64_t nblocks, uint32_t d, const uint64_t* probe, uint64_t* scores_ct,
                          uint64_t* ws, int* err, cudaStream_t st, cudaEvent_t* ev) {
    if (nblocks == 0) return cudaSuccess;
    uint64_t nl = 0;
    constexpr int NB = 2;
    uint64_t* X = ws;
    uint64_t* C = X + nblocks * 15 * N;
    uint64_t* KS = C + nblocks * 6 * N;
    uint64_t* O = X;
    // grid.z is limited to 65535: process at most 65535 groups / blocks per pass
    const uint64_t max_z = 65535;
    if (ev) cudaEventRecord(ev[0], st);
    constexpr int STAGES = 6;
    const int smem = STAGES * (2 + 2 * NB) * TT * 8;
    cudaError_t ea = cudaFuncSetAttribute(k_tensor_tma<NB, STAGES>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (ea != cudaSuccess) return ea;
    for (uint64_t g0 = 0; g0 < nblocks; g0 += max_z * NB) {
        const uint64_t nb = nblocks - g0 < max_z * NB ? nblocks - g0 : max_z * NB;
        dim3 grid(N / TT, 5, (unsigned)((nb + NB - 1) / NB));
        k_tensor_tma<NB, STAGES><<<grid, TT + 32, smem, st>>>(gallery + g0 * d * 10 * N, probe,
                                                               X + g0 * 15 * N, nb, d, err);
        nl++;
    }
    if (ev) cudaEventRecord(ev[1], st);
    const uint64_t chunk = 1u << 30;
    for (uint64_t off = 0; off < nblocks * 15; off += chunk) {
        const uint64_t n = nblocks * 15 - off < chunk ? nblocks * 15 - off : chunk;
        k_ntt_batch<true><<<(unsigned)n, NTT_THREADS, N * 8, st>>>(tw, X + off * N, 5, 0);
        nl++;
    }
    if (ev) cudaEventRecord(ev[2], st);
    for (uint64_t b0 = 0; b0 < nblocks; b0 += max_z) {
        const uint64_t nb = nblocks - b0 < max_z ? nblocks - b0 : max_z;
        k_scale_round<<<dim3(N / 256, 3, (unsigned)nb), 256, 0, st>>>(X + b0 * 15 * N, C + b0 * 6 * N,
                                                                     KS + b0 * 4 * N);
        nl++;
    }
    if (ev) cudaEventRecord(ev[3], st);
    for (uint64_t off = 0; off < nblocks * 4; off += chunk) {
        const uint64_t n = nblocks * 4 - off < chunk ? nblocks * 4 - off : chunk;
        k_ntt_batch<false><<<(unsigned)n, NTT_THREADS, N * 8, st>>>(tw, KS + off * N, 2, 0);
        nl++;
    }
    for (uint64_t b0 = 0; b0 < nblocks; b0 += max_z) {
        const uint64_t nb = nblocks - b0 < max_z ? nblocks - b0 : max_z;
        k_ks_mul<<<dim3(N / 256, 2, (unsigned)nb), 256, 0, st>>>(KS + b0 * 4 * N, k.evk_ntt,
                                                                 O + b0 * 4 * N);
        nl++;
    }
    for (uint64_t off = 0; off < nblocks * 4; off += chunk) {
        const uint64_t n = nblocks * 4 - off < chunk ? nblocks * 4 - off : chunk;
        k_ntt_batch<true><<<(unsigned)n, NTT_THREADS, N * 8, st>>>(tw, O + off * N, 2, 0);
        nl++;
    }
    for (uint64_t b0 = 0; b0 < nblocks; b0 += max_z) {
        const uint64_t nb = nblocks - b0 < max_z ? nblocks - b0 : max_z;
        k_ks_finish<<<dim3(N / 256, 4, (unsigned)nb), 256, 0, st>>>(C + b0 * 6 * N, O + b0 * 4 * N,
                                                                    scores_ct + b0 * 4 * N);
        nl++;
    }
    if (ev) cudaEventRecord(ev[4], st);
    count_launches(nl);
    return cudaGetLastError();
}

}  // namespace hers
