// Batched Shield-MPPI: B independent control problems with their own K_i, T_i,
// track and state, one closed-loop update of all of them in ONE persistent
// launch over a device work queue (Alg. 2 body per problem).
//
// Work items are (problem i, chunk c) pairs of 2 RB rollouts (two per thread,
// packed FP32 pairs, when C = 1.5 and |steer| <= 1/2; else RB), ordered by
// decreasing horizon T_i so that the problems with the longest repairs finish
// their rollouts first.  A grid of #SMs x (blocks per SM) blocks pops items
// from an atomic head.  A block stages the problem's segment-pair table (bulk
// copy) and nominal controls, finds the nearest segment of x0, runs the item's
// rollouts (the same per-rollout code as the single-problem kernel), writes
// the costs and the chunk minimum, and takes a ticket on the problem's
// completion counter.  The block that completes the last chunk of problem i
// then, in place and while other blocks keep popping rollout items:
//   - forms V+ (Eq. 10-11): global minimum over the chunk minima, weights for
//     all K_i costs, noise regenerated for the rollouts with weight above
//     w_skip (bound <= 1e-8 on V+), per-thread float sums, float64 normaliser;
//   - repairs V+ into V_safe (Alg. 1 with Armijo backtracking, repair_in_block);
//   - executes v_0^safe on the disturbed system (Eq. 26) and warm-starts
//     V <- shift(V+).
// Randomness per problem: Philox counter word (stream | i << 8).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <string>
#include <vector>

#include "rollout2.cuh"
#include "shield.cuh"

using namespace smppi;

namespace smppi {

struct BatchInst {
    int K, T, N_r, n_track;
    int rec_off;       // first float4 of this problem's segment-pair table
    int V_off;         // first control of this problem in V / V_safe
    int S_off;         // first cost of this problem in S
    int chunk_off;     // first chunk of this problem in chunk_min
    int n_chunks;
    float w2, qd_w2, w_skip;
};

struct BatchArgs {
    const BatchInst* inst;
    const int2* items;
    int n_items;
    const float4* rec;     // segment-pair tables, per-problem offsets
    float* S;
    float* chunk_min;
    unsigned* done;        // [B] completion counters (0 on entry, left 0)
    unsigned* head;        // work-queue head (0 on entry)
    float* x0;             // [B][6]
    float* V;              // controls, per-problem offsets
    float* V_safe;
    uint32_t iter;
    const uint32_t* iter_dev;
    int n_repair, ck;
    int n_track_max, T_max;
    unsigned* status;
    unsigned* viol;        // [B] executed steps violating the DCBF condition (monitor)
    unsigned* outside;     // [B] executed steps ending outside the track (monitor)
};

constexpr int BATCH_PPT = 8;      // costs per thread in one pass of the problem update
constexpr int BATCH_MAXPS = 4;    // pair sets per thread (pairs <= 4 * RB)

// FAST (C = 1.5, |steer| <= 1/2): a work item is 2 RB rollouts, two per
// thread on the packed path (rollout2.cuh); otherwise RB, one per thread.
template <int RB, bool FAST>
__global__ void __launch_bounds__(RB, 1) batch_kernel(DevParams P0, BatchArgs a) {
    constexpr int NW = RB / 32;
    constexpr int CHUNK = FAST ? 2 * RB : RB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nmax = a.n_track_max, Tm = a.T_max;
    float4* rec = reinterpret_cast<float4*>(smem_raw);
    float4* Vs4 = rec + 3 * (nmax + 5);                     // V rows of the rollouts (2 Tm float4)
    float2* Vs = reinterpret_cast<float2*>(Vs4 + 2 * Tm);   // nominal V, then V+
    float2* Vw = Vs + Tm;                                      // repaired controls
    float2* G = Vw + Tm;
    float* tape_s = reinterpret_cast<float*>(G + Tm);
    int* l_k = reinterpret_cast<int*>(tape_s + (size_t)(Tm + 2) * NFIELD);
    float* l_w = reinterpret_cast<float*>(l_k + RB * BATCH_PPT);
    float* acc_s = l_w + RB * BATCH_PPT;                       // [2 Tm]
    const GradWs gws = grad_ws_at(reinterpret_cast<unsigned char*>(acc_s + 2 * Tm), Tm);
    __shared__ __align__(8) uint64_t bar;
    __shared__ RepairSmem rsm;
    __shared__ float red_f[NW];
    __shared__ int red_i[NW];
    __shared__ int w_cnt[NW];
    __shared__ int s_item, s_last;
    __shared__ double s_eta;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t iter = a.iter + (a.iter_dev ? *a.iter_dev : 0u);
    if (tid == 0) mbar_init(&bar, 1);
    __syncthreads();
    uint32_t phase = 0;
    int staged = -1, s0 = 0;
    float d20 = 0.0f;

    for (;;) {
        // after any block of the launch (or of an earlier replay not yet read by
        // the host) gave up on a bounded wait, no block takes further items: the
        // launch then ends within one item's time instead of every later item
        // waiting out its own limit
        if (tid == 0)
            s_item = (*reinterpret_cast<volatile unsigned*>(a.status) & SMPPI_DEV_TIMEOUT)
                         ? a.n_items
                         : (int)atomicAdd(a.head, 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= a.n_items) break;
        const int2 ic = a.items[item];
        const int i = ic.x, c = ic.y;
        const BatchInst D = a.inst[i];
        DevParams P = P0;
        P.K = D.K; P.T = D.T; P.N_r = D.N_r; P.n_track = D.n_track;
        P.w2 = D.w2; P.qd_w2 = D.qd_w2; P.w_skip = D.w_skip;
        const int T = D.T, n = D.n_track;
        const uint32_t ctr3 = (uint32_t)i << 8;
        State x = make_state(a.x0 + 6 * i);
        if (staged != i) {
            // stage the problem's track (bulk copy), its nominal controls, nearest segment
            if (tid == 0) {
                const uint32_t bytes = (uint32_t)rec_table_bytes(n);
                mbar_expect_tx(&bar, bytes);
                bulk_g2s(rec, a.rec + D.rec_off, bytes, &bar);
            }
            const float2* Vg = reinterpret_cast<const float2*>(a.V) + D.V_off;
            for (int t = tid; t < T; t += RB) {
                const float2 v = Vg[t];
                Vs[t] = v;
                const float g0 = P.gis0 * v.x, g1 = P.gis1 * v.y;
                if (FAST) {   // broadcast pairs of the packed rollouts
                    Vs4[2 * t] = make_float4(v.x, v.x, v.y, v.y);
                    Vs4[2 * t + 1] = make_float4(g0, g0, g1, g1);
                } else {
                    Vs4[t] = make_float4(v.x, v.y, g0, g1);
                }
            }
            // thread 0 has armed the barrier (arrive.expect_tx) before any thread
            // of the block, its own warp's lanes included, starts to wait on it
            __syncthreads();
            // a failed wait ends the whole block (block-uniform decision), after
            // thread 0 has let the copy in flight land
            const bool ok = mbar_wait_bounded(&bar, phase);
            if (__syncthreads_or(!ok)) {
                if (tid == 0) {
                    atomicOr(a.status, SMPPI_DEV_TIMEOUT);
                    mbar_wait_bounded(&bar, phase);
                }
                return;
            }
            phase ^= 1u;
            s0 = block_nearest_segment<RB>(rec, n, x.X, x.Y, red_f, red_i, &d20, a.status);
            staged = i;
        }

        // CHUNK rollouts of problem i (the single-problem rollout code)
        float m = 3.0e38f;
        if (FAST) {
            const int ka = c * CHUNK + tid, kb = ka + RB;
            if (ka < D.K) {
                const float2 S2 = x2::rollout2<false>(P, rec, Vs4, x, s0, d20, (uint32_t)ka,
                                                      (uint32_t)kb, iter, ctr3, nullptr, nullptr);
                a.S[D.S_off + ka] = S2.x;
                if (!isfinite(S2.x)) atomicOr(a.status, SMPPI_DEV_NUMERIC);
                m = S2.x;
                if (kb < D.K) {
                    a.S[D.S_off + kb] = S2.y;
                    if (!isfinite(S2.y)) atomicOr(a.status, SMPPI_DEV_NUMERIC);
                    m = fminf(m, S2.y);
                }
            }
        } else {
            const int k = c * CHUNK + tid;
            if (k < D.K) {
                const float S = rollout_sample<false, false>(P, rec, Vs4, x, s0, d20, (uint32_t)k,
                                                             iter, ctr3, nullptr);
                a.S[D.S_off + k] = S;
                if (!isfinite(S)) atomicOr(a.status, SMPPI_DEV_NUMERIC);
                m = S;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) red_f[warp] = m;
        __syncthreads();
        if (tid == 0) {
            float mb = red_f[0];
            for (int w = 1; w < NW; ++w) mb = fminf(mb, red_f[w]);
            a.chunk_min[D.chunk_off + c] = mb;
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) s_last = (atomicAdd(&a.done[i], 1u) == (unsigned)D.n_chunks - 1u);
        __syncthreads();
        if (!s_last) continue;

        // ---- this block completed problem i: softmin update (Eq. 10-11) ----
        __threadfence();
        float mm = 3.0e38f;
        for (int b = tid; b < D.n_chunks; b += RB) mm = fminf(mm, __ldcg(&a.chunk_min[D.chunk_off + b]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mm = fminf(mm, __shfl_xor_sync(0xffffffffu, mm, o));
        if (lane == 0) red_f[warp] = mm;
        __syncthreads();
        mm = red_f[0];
        for (int w = 1; w < NW; ++w) mm = fminf(mm, red_f[w]);
        const int npair = (T + 1) >> 1;
        const int C = npair <= RB ? RB / npair : 1;            // slots per pair
        const int cslot = npair <= RB ? tid / npair : 0;
        const int pbase = npair <= RB ? tid % npair : tid;
        const bool worker = cslot < C;
        float ac[BATCH_MAXPS][4];
#pragma unroll
        for (int u = 0; u < BATCH_MAXPS; ++u) ac[u][0] = ac[u][1] = ac[u][2] = ac[u][3] = 0.0f;
        float eta_t = 0.0f;
        for (int kb = 0; kb < D.K; kb += RB * BATCH_PPT) {
            float om[BATCH_PPT];
            int ntake = 0;
#pragma unroll
            for (int u = 0; u < BATCH_PPT; ++u) {
                const int kk = kb + tid * BATCH_PPT + u;
                om[u] = kk < D.K ? expf((mm - __ldcg(&a.S[D.S_off + kk])) * P.lam_inv) : 0.0f;
                eta_t += om[u];
                ntake += om[u] > P.w_skip;
            }
            int incl = ntake;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            if (lane == 31) w_cnt[warp] = incl;
            __syncthreads();
            int off = incl - ntake, tot = 0;
            for (int w = 0; w < NW; ++w) {
                if (w < warp) off += w_cnt[w];
                tot += w_cnt[w];
            }
#pragma unroll
            for (int u = 0; u < BATCH_PPT; ++u)
                if (om[u] > P.w_skip) {
                    l_k[off] = kb + tid * BATCH_PPT + u;
                    l_w[off] = om[u];
                    ++off;
                }
            __syncthreads();
            if (worker) {
                for (int li = cslot; li < tot; li += C) {
#pragma unroll
                    for (int u = 0; u < BATCH_MAXPS; ++u) {
                        const int p = pbase + u * RB;
                        if (u > 0 && npair <= RB) break;
                        if (p >= npair) break;
                        const uint4 r = philox10(make_uint4((uint32_t)l_k[li], (uint32_t)p, iter, ctr3), P);
                        const float2 ze = box_muller(r.x, r.y), zo = box_muller(r.z, r.w);
                        const float w0 = l_w[li] * P.sig0, w1 = l_w[li] * P.sig1;
                        ac[u][0] = fmaf(w0, ze.x, ac[u][0]);
                        ac[u][1] = fmaf(w1, ze.y, ac[u][1]);
                        ac[u][2] = fmaf(w0, zo.x, ac[u][2]);
                        ac[u][3] = fmaf(w1, zo.y, ac[u][3]);
                    }
                }
            }
            __syncthreads();
        }
        // normaliser: per-warp float sums, float64 across warps
        float ef = eta_t;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ef += __shfl_xor_sync(0xffffffffu, ef, o);
        if (lane == 0) red_f[warp] = ef;
        for (int j = tid; j < 2 * T; j += RB) acc_s[j] = 0.0f;
        __syncthreads();
        if (tid == 0) {
            double e = 0.0;
            for (int w = 0; w < NW; ++w) e += (double)red_f[w];
            s_eta = 1.0 / e;
        }
        for (int cc = 0; cc < C; ++cc) {
            if (worker && cslot == cc) {
#pragma unroll
                for (int u = 0; u < BATCH_MAXPS; ++u) {
                    const int p = pbase + u * RB;
                    if (u > 0 && npair <= RB) break;
                    if (p >= npair) break;
                    acc_s[4 * p] += ac[u][0];
                    acc_s[4 * p + 1] += ac[u][1];
                    if (2 * p + 1 < T) {
                        acc_s[4 * p + 2] += ac[u][2];
                        acc_s[4 * p + 3] += ac[u][3];
                    }
                }
            }
            __syncthreads();
        }
        const double inv_eta = s_eta;
        float2* Vg = reinterpret_cast<float2*>(a.V) + D.V_off;
        for (int t = tid; t < T; t += RB) {
            const float2 v = Vs[t];
            const float vx = clampf((float)fma((double)acc_s[2 * t], inv_eta, (double)v.x), P.umin0, P.umax0);
            const float vy = clampf((float)fma((double)acc_s[2 * t + 1], inv_eta, (double)v.y), P.umin1, P.umax1);
            Vs[t] = make_float2(vx, vy);     // V+
            Vw[t] = Vs[t];
        }
        __syncthreads();
        // ---- safety shield on V+ (Alg. 1) ----
        State xr = make_state(a.x0 + 6 * i);
        if (a.n_repair > 0)
            repair_in_block<RB, FAST>(P, rec, xr, s0, Vw, G, tape_s, a.n_repair, 1, 0.0f, a.ck,
                                nullptr, nullptr, a.status, rsm, NoSide(), &gws);
        float2* Vsafe = reinterpret_cast<float2*>(a.V_safe) + D.V_off;
        for (int t = tid; t < T; t += RB) Vsafe[t] = Vw[t];
        // ---- closed loop: x0 <- f(x0, v0_safe) + w (Eq. 26), V <- shift(V+) ----
        if (tid == 0) {
            State xn = xr;
            const float2 v0 = Vw[0];
            model_step(P, xn, clampf(v0.x, P.umin0, P.umax0), clampf(v0.y, P.umin1, P.umax1));
            const uint4 r = philox10(make_uint4(0u, 0u, iter, ctr3 | 1u), P);
            const float2 z = box_muller(r.x, r.y);
            float* xo = a.x0 + 6 * i;
            xo[0] = xn.vx;
            xo[1] = fmaf(P.dsig0, z.x, xn.vy);
            xo[2] = fmaf(P.dsig1, z.y, xn.r);
            xo[3] = xn.X;
            xo[4] = xn.Y;
            xo[5] = xn.psi;
            a.done[i] = 0u;
            // safety monitor of the executed step: h = w^2 - e_y^2 (Eq. 23) of x0 and of the
            // new state (tracked from x0's segment), DCBF condition of Eq. 17
            float d21;
            bool nofb = false;
            walk_rec<false>(rec, n, s0, xn.X, xn.Y, d21, nofb);
            const float h0 = P.w2 - d20, h1 = P.w2 - d21;
            if (h1 < P.one_m_alpha * h0) a.viol[i] += 1u;
            if (h1 < 0.0f) a.outside[i] += 1u;
        }
        for (int t = tid; t < T; t += RB) Vg[t] = Vs[t + 1 < T ? t + 1 : T - 1];
        staged = -1;      // Vs now holds V+ of this problem
        __syncthreads();
    }
}

// Advance the update counter of graph replays.
__global__ void batch_iter_inc(uint32_t* iter_dev) { *iter_dev += 1u; }

// Segment-pair tables of all problems (layout in device.cuh); block i builds
// problem i's n_i + 5 records at rec + rec_off.
__global__ void batch_rec_tables(const float* __restrict__ xy, const BatchInst* __restrict__ inst,
                                 const int* __restrict__ track_off, int B, float4* __restrict__ rec) {
    const int i = blockIdx.x;
    if (i >= B) return;
    const BatchInst D = inst[i];
    const int n = D.n_track;
    const float* p = xy + 2 * (size_t)track_off[i];
    float4* r = rec + D.rec_off;
    for (int j = threadIdx.x; j < n + 5; j += blockDim.x) {
        float ax[2], ay[2], dx[2], dy[2], gx[2], gy[2];
        for (int h = 0; h < 2; ++h) {
            const int a0 = (j - 1 + h + n) % n, a1 = (a0 + 1 == n) ? 0 : a0 + 1;
            ax[h] = p[2 * a0];
            ay[h] = p[2 * a0 + 1];
            dx[h] = p[2 * a1] - ax[h];
            dy[h] = p[2 * a1 + 1] - ay[h];
            const float l2 = fmaf(dx[h], dx[h], dy[h] * dy[h]);
            const float iv = l2 > 0.0f ? 1.0f / l2 : 0.0f;
            gx[h] = dx[h] * iv;
            gy[h] = dy[h] * iv;
        }
        r[3 * j] = make_float4(-ax[0], -ax[1], -ay[0], -ay[1]);
        r[3 * j + 1] = make_float4(-dx[0], -dx[1], -dy[0], -dy[1]);
        r[3 * j + 2] = make_float4(gx[0], gx[1], gy[0], gy[1]);
    }
}

}  // namespace smppi

// ============================================================================
// Host side: C ABI of the batch
// ============================================================================
struct smppi_batch {
    smppi_params shared;
    DevParams dp;
    int B = 0;
    std::vector<smppi_instance_desc> desc;
    std::vector<BatchInst> inst;          // host copy (offsets depend on RB)
    BatchInst* d_inst = nullptr;
    int* d_track_off = nullptr;
    int2* d_items = nullptr;
    int n_items = 0, max_items = 0;
    float4* rec = nullptr;                // segment-pair tables of all problems
    float* S = nullptr;
    float* chunk_min = nullptr;
    unsigned* done = nullptr;
    unsigned* head = nullptr;
    unsigned* status = nullptr;
    unsigned* viol = nullptr;             // [B] safety-monitor counters
    unsigned* outside = nullptr;
    uint32_t* iter_dev = nullptr;
    float* tune_x0 = nullptr;             // scratch state for the autotuner
    float* tune_V = nullptr;
    float* tune_Vs = nullptr;
    int V_len = 0;                        // floats spanned by V
    int RB = 0, bps = 0, grid = 0;        // rollouts per item, blocks per SM, grid
    bool tuned = false;
    int T_max = 0, n_track_max = 0, ck = 0, sms = 1;
    cudaStream_t st = nullptr, cap = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::string graph_key, err;
};

namespace {

// the message of the last failure outside a batch handle, per host thread
thread_local std::string g_batch_err;

smppi_status bfail(smppi_batch* b, smppi_status s, const std::string& m) {
    if (b) b->err = m;
    else g_batch_err = m;
    return s;
}

#define BCU(b, call)                                                                       \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return bfail((b), SMPPI_ERR_CUDA,                                              \
                         std::string(#call) + ": " + cudaGetErrorString(e_));              \
    } while (0)

size_t batch_smem(int RB, int n_track_max, int T_max) {
    return rec_table_bytes(n_track_max) + (size_t)T_max * 32 + (size_t)T_max * 8 * 3 +
           (size_t)(T_max + 2) * NFIELD * 4 + (size_t)RB * BATCH_PPT * 8 + (size_t)T_max * 2 * 4 +
           grad_ws_bytes(T_max);
}

template <bool FAST>
const void* batch_kernel_ptr_t(int RB) {
    if (RB == 64) return (const void*)batch_kernel<64, FAST>;
    if (RB == 256) return (const void*)batch_kernel<256, FAST>;
    return (const void*)batch_kernel<128, FAST>;
}

// The branch-free model step applies when C = 1.5 and the steering bound keeps
// |delta| <= 0.5 (same selection as the single-problem rollout).
bool batch_fast(const smppi_batch* b) { return b->dp.tyre15 && b->dp.steer_small; }

const void* batch_kernel_ptr(const smppi_batch* b, int RB) {
    return batch_fast(b) ? batch_kernel_ptr_t<true>(RB) : batch_kernel_ptr_t<false>(RB);
}

// Offsets, chunk counts and the work-item order (decreasing T, then problem,
// then chunk) for items of RB threads (2 RB rollouts on the packed path).
smppi_status layout(smppi_batch* b, int RB) {
    std::vector<int> order(b->B);
    for (int i = 0; i < b->B; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return b->desc[x].T > b->desc[y].T; });
    const int chunk = batch_fast(b) ? 2 * RB : RB;
    int S_off = 0, chunk_off = 0;
    std::vector<int2> items;
    for (int i = 0; i < b->B; ++i) {
        BatchInst& D = b->inst[i];
        D.S_off = S_off;
        D.n_chunks = (D.K + chunk - 1) / chunk;
        D.chunk_off = chunk_off;
        S_off += D.K;
        chunk_off += D.n_chunks;
    }
    for (int i : order)
        for (int c = 0; c < b->inst[i].n_chunks; ++c) items.push_back(make_int2(i, c));
    if ((int)items.size() > b->max_items) return bfail(b, SMPPI_ERR_ARG, "work items exceed capacity");
    b->n_items = (int)items.size();
    BCU(b, cudaMemcpyAsync(b->d_inst, b->inst.data(), sizeof(BatchInst) * b->B,
                           cudaMemcpyHostToDevice, b->st));
    BCU(b, cudaMemcpyAsync(b->d_items, items.data(), sizeof(int2) * items.size(),
                           cudaMemcpyHostToDevice, b->st));
    BCU(b, cudaStreamSynchronize(b->st));
    b->RB = RB;
    return SMPPI_OK;
}

smppi_status enqueue_batch(smppi_batch* b, cudaStream_t st, float* x0, float* V, float* Vs,
                           uint32_t iter, int n_repair, uint32_t* iter_dev) {
    BatchArgs a;
    a.inst = b->d_inst; a.items = b->d_items; a.n_items = b->n_items;
    a.rec = b->rec; a.S = b->S; a.chunk_min = b->chunk_min;
    a.done = b->done; a.head = b->head;
    a.x0 = x0; a.V = V; a.V_safe = Vs;
    a.iter = iter; a.iter_dev = iter_dev;
    a.n_repair = n_repair; a.ck = b->ck;
    a.n_track_max = b->n_track_max; a.T_max = b->T_max;
    a.status = b->status;
    a.viol = b->viol;
    a.outside = b->outside;
    const size_t smem = batch_smem(b->RB, b->n_track_max, b->T_max);
    BCU(b, cudaMemsetAsync(b->head, 0, sizeof(unsigned), st));
    BCU(b, ensure_smem(batch_kernel_ptr(b, b->RB), smem));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(b->grid);
    cfg.blockDim = dim3(b->RB);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    void* args[] = {(void*)&b->dp, (void*)&a};
    BCU(b, cudaLaunchKernelExC(&cfg, batch_kernel_ptr(b, b->RB), args));
    BCU(b, cudaGetLastError());
    return SMPPI_OK;
}

// Blocks per SM the kernel can keep resident for RB (0 if it does not fit).
int max_bps(smppi_batch* b, int RB) {
    int nb = 0;
    const size_t smem = batch_smem(RB, b->n_track_max, b->T_max);
    if (ensure_smem(batch_kernel_ptr(b, RB), smem) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_kernel_ptr(b, RB), RB, smem) !=
        cudaSuccess)
        return 0;
    return nb;
}

// Autotuner: time one closed-loop update of every candidate (rollouts per item
// x blocks per SM) on a scratch copy of the state and keep the fastest.
smppi_status autotune(smppi_batch* b, const float* x0, const float* V, const float* Vs,
                      int n_repair) {
    struct Cand { int RB, bps; };
    std::vector<Cand> cands;
    for (int RB : {64, 128, 256}) {
        if ((b->T_max + 1) / 2 > BATCH_MAXPS * RB) continue;
        const int mb = max_bps(b, RB);
        if (mb < 1) continue;
        for (int bps : {mb, std::max(1, mb / 2)}) {
            bool dup = false;
            for (auto& c : cands) dup |= (c.RB == RB && c.bps == bps);
            if (!dup) cands.push_back({RB, bps});
        }
    }
    if (cands.empty()) return bfail(b, SMPPI_ERR_ARG, "no launch shape fits this batch");
    cudaEvent_t e0, e1;
    BCU(b, cudaEventCreate(&e0));
    BCU(b, cudaEventCreate(&e1));
    float best = 3.0e38f;
    Cand pick = cands[0];
    for (const Cand& c : cands) {
        smppi_status s = layout(b, c.RB);
        if (s != SMPPI_OK) return s;
        b->bps = c.bps;
        b->grid = b->sms * c.bps;
        float t_c = 0.0f;
        for (int rep = 0; rep < 2; ++rep) {
            BCU(b, cudaMemcpyAsync(b->tune_x0, x0, sizeof(float) * 6 * b->B, cudaMemcpyDeviceToDevice, b->st));
            BCU(b, cudaMemcpyAsync(b->tune_V, V, sizeof(float) * b->V_len, cudaMemcpyDeviceToDevice, b->st));
            BCU(b, cudaMemcpyAsync(b->tune_Vs, Vs, sizeof(float) * b->V_len, cudaMemcpyDeviceToDevice, b->st));
            BCU(b, cudaEventRecord(e0, b->st));
            s = enqueue_batch(b, b->st, b->tune_x0, b->tune_V, b->tune_Vs, 0u, n_repair, nullptr);
            if (s != SMPPI_OK) return s;
            BCU(b, cudaEventRecord(e1, b->st));
            BCU(b, cudaEventSynchronize(e1));
            float ms = 0.0f;
            BCU(b, cudaEventElapsedTime(&ms, e0, e1));
            if (rep == 1) t_c = ms;      // the first run warms up
        }
        if (t_c < best) { best = t_c; pick = c; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    smppi_status s = layout(b, pick.RB);
    if (s != SMPPI_OK) return s;
    b->bps = pick.bps;
    b->grid = b->sms * pick.bps;
    b->tuned = true;
    BCU(b, cudaMemsetAsync(b->status, 0, sizeof(unsigned), b->st));
    // the timing runs stepped scratch copies: they do not count for the monitor
    BCU(b, cudaMemsetAsync(b->viol, 0, sizeof(unsigned) * b->B, b->st));
    BCU(b, cudaMemsetAsync(b->outside, 0, sizeof(unsigned) * b->B, b->st));
    return SMPPI_OK;
}

void bfree(smppi_batch* b) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    void* ptrs[] = {b->d_inst, b->d_track_off, b->d_items, b->rec, b->S, b->chunk_min,
                    b->done, b->head, b->status, b->viol, b->outside, b->iter_dev,
                    b->tune_x0, b->tune_V, b->tune_Vs};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (b->cap) cudaStreamDestroy(b->cap);
}

}  // namespace

extern "C" {

smppi_status smppi_batch_create(const smppi_params* shared, int B, const smppi_instance_desc* desc,
                                const float* tracks_xy, int block_rollouts, void* cuda_stream,
                                smppi_batch** out) {
    if (!out) return bfail(nullptr, SMPPI_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!shared || !desc || !tracks_xy) return bfail(nullptr, SMPPI_ERR_ARG, "NULL argument");
    if (B < 1 || B > (1 << 24)) return bfail(nullptr, SMPPI_ERR_ARG, "B must be in [1, 2^24]");
    if (block_rollouts != 0 && block_rollouts != 64 && block_rollouts != 128 && block_rollouts != 256)
        return bfail(nullptr, SMPPI_ERR_ARG, "block_rollouts must be 0, 64, 128 or 256");
    // the shared parameters are checked with a placeholder problem size
    smppi_params chk = *shared;
    chk.K = 1; chk.T = 1; chk.N_r = 0; chk.n_track = 3; chk.track_xy = tracks_xy;
    chk.half_width = 1.0f; chk.max_seq = 1;
    smppi_status s = validate_params(&chk);
    if (s != SMPPI_OK) return bfail(nullptr, s, "shared parameters rejected");
    if (shared->state_kind != 0) return bfail(nullptr, SMPPI_ERR_ARG, "the batch needs state_kind 0");
    smppi_batch* b = new smppi_batch();
    b->shared = *shared;
    b->B = B;
    b->desc.assign(desc, desc + B);
    b->st = static_cast<cudaStream_t>(cuda_stream);
    b->inst.resize(B);
    long long totK = 0, rec_tot = 0, chunks64 = 0;
    std::vector<int> track_off(B);
    for (int i = 0; i < B; ++i) {
        const smppi_instance_desc& d = desc[i];
        if (d.K < 1 || d.K > (1 << 22) || d.T < 1 || d.T > SMPPI_MAX_T || d.N_r < 0 || d.N_r > d.T ||
            d.n_track < 3 || d.n_track > SMPPI_MAX_TRACK || !(d.half_width > 0.0f) ||
            d.track_offset < 0 || d.V_offset < 0) {
            delete b;
            return bfail(nullptr, SMPPI_ERR_ARG, "instance descriptor " + std::to_string(i) + " out of range");
        }
        BatchInst& D = b->inst[i];
        D.K = d.K; D.T = d.T; D.N_r = d.N_r; D.n_track = d.n_track;
        D.rec_off = (int)rec_tot;
        D.V_off = d.V_offset;
        const double w2 = (double)d.half_width * d.half_width;
        D.w2 = (float)w2;
        D.qd_w2 = (float)(shared->q_d / w2);
        const double e_max = std::max(shared->sigma[0], shared->sigma[1]) * std::sqrt(48.0 * std::log(2.0));
        D.w_skip = e_max > 0.0 ? (float)(1e-8 / ((double)d.K * e_max)) : 3.0e38f;
        rec_tot += 3LL * (d.n_track + 5);
        totK += d.K;
        chunks64 += (d.K + 63) / 64;
        track_off[i] = d.track_offset;
        b->T_max = std::max(b->T_max, d.T);
        b->n_track_max = std::max(b->n_track_max, d.n_track);
        b->V_len = std::max(b->V_len, 2 * (d.V_offset + d.T));
    }
    smppi_params pp = *shared;
    pp.K = 1; pp.T = b->T_max; pp.N_r = b->T_max; pp.half_width = 1.0f;
    b->dp = derive_params(pp);
    b->ck = shared->checkpoint > 0 ? shared->checkpoint : (int)std::ceil(std::sqrt((double)b->T_max));
    b->max_items = (int)chunks64;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    if (b->sms < 1) b->sms = 1;
    cudaError_t e = cudaSuccess;
#define BALLOC(ptr, bytes) if (e == cudaSuccess) e = cudaMalloc((void**)&(ptr), std::max<size_t>(16, (bytes)));
    BALLOC(b->d_inst, sizeof(BatchInst) * B);
    BALLOC(b->d_track_off, sizeof(int) * B);
    BALLOC(b->d_items, sizeof(int2) * b->max_items);
    BALLOC(b->rec, sizeof(float4) * rec_tot);
    BALLOC(b->S, sizeof(float) * totK);
    BALLOC(b->chunk_min, sizeof(float) * chunks64);
    BALLOC(b->done, sizeof(unsigned) * B);
    BALLOC(b->head, sizeof(unsigned));
    BALLOC(b->status, sizeof(unsigned));
    BALLOC(b->viol, sizeof(unsigned) * B);
    BALLOC(b->outside, sizeof(unsigned) * B);
    BALLOC(b->iter_dev, sizeof(uint32_t));
    BALLOC(b->tune_x0, sizeof(float) * 6 * B);
    BALLOC(b->tune_V, sizeof(float) * b->V_len);
    BALLOC(b->tune_Vs, sizeof(float) * b->V_len);
#undef BALLOC
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->done, 0, sizeof(unsigned) * B, b->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->status, 0, sizeof(unsigned), b->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->viol, 0, sizeof(unsigned) * B, b->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->outside, 0, sizeof(unsigned) * B, b->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->iter_dev, 0, sizeof(uint32_t), b->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_track_off, track_off.data(), sizeof(int) * B, cudaMemcpyHostToDevice, b->st);
    if (e != cudaSuccess) {
        const bool oom = e == cudaErrorMemoryAllocation;
        bfail(nullptr, oom ? SMPPI_ERR_NOMEM : SMPPI_ERR_CUDA, cudaGetErrorString(e));
        bfree(b);
        delete b;
        return oom ? SMPPI_ERR_NOMEM : SMPPI_ERR_CUDA;
    }
    s = layout(b, block_rollouts ? block_rollouts : 128);
    if (s == SMPPI_OK) {
        batch_rec_tables<<<B, 128, 0, b->st>>>(tracks_xy, b->d_inst, b->d_track_off, B, b->rec);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
        if (e != cudaSuccess) s = bfail(nullptr, SMPPI_ERR_CUDA, cudaGetErrorString(e));
    } else {
        g_batch_err = b->err;
    }
    if (s == SMPPI_OK && block_rollouts) {
        const int mb = max_bps(b, block_rollouts);
        if (mb < 1) s = bfail(nullptr, SMPPI_ERR_ARG, "block_rollouts does not fit this batch");
        b->bps = mb;
        b->grid = b->sms * mb;
        b->tuned = true;
    }
    if (s != SMPPI_OK) {
        bfree(b);
        delete b;
        return s;
    }
    *out = b;
    return SMPPI_OK;
}

smppi_status smppi_batch_destroy(smppi_batch* b) {
    if (!b) return SMPPI_OK;
    cudaStreamSynchronize(b->st);
    bfree(b);
    delete b;
    return SMPPI_OK;
}

const char* smppi_batch_last_error(const smppi_batch* b) {
    return b ? b->err.c_str() : g_batch_err.c_str();
}

smppi_status smppi_batch_step(smppi_batch* b, float* x0, float* V, float* V_safe, uint32_t iter,
                              int n_repair) {
    if (!b) return bfail(nullptr, SMPPI_ERR_ARG, "batch is NULL");
    if (!x0 || !V || !V_safe) return bfail(b, SMPPI_ERR_ARG, "x0, V, V_safe must not be NULL");
    if (n_repair < 0 || n_repair > 100000) return bfail(b, SMPPI_ERR_ARG, "n_repair in [0, 1e5]");
    if (!b->tuned) {
        smppi_status s = autotune(b, x0, V, V_safe, n_repair);
        if (s != SMPPI_OK) return s;
    }
    return enqueue_batch(b, b->st, x0, V, V_safe, iter, n_repair, nullptr);
}

smppi_status smppi_batch_loop(smppi_batch* b, float* x0, float* V, float* V_safe, uint32_t iter0,
                              int n_repair, int n_updates) {
    if (!b) return bfail(nullptr, SMPPI_ERR_ARG, "batch is NULL");
    if (!x0 || !V || !V_safe) return bfail(b, SMPPI_ERR_ARG, "x0, V, V_safe must not be NULL");
    if (n_repair < 0 || n_repair > 100000 || n_updates < 0)
        return bfail(b, SMPPI_ERR_ARG, "n_repair in [0, 1e5], n_updates >= 0");
    if (!b->tuned) {
        smppi_status s = autotune(b, x0, V, V_safe, n_repair);
        if (s != SMPPI_OK) return s;
    }
    char key[256];
    std::snprintf(key, sizeof(key), "%p %p %p %u %d %d %d", (void*)x0, (void*)V, (void*)V_safe,
                  iter0, n_repair, b->RB, b->grid);
    if (!b->gexec || b->graph_key != key) {
        if (b->gexec) {
            cudaGraphExecDestroy(b->gexec);
            b->gexec = nullptr;
        }
        cudaGraph_t g = nullptr;
        BCU(b, cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
        smppi_status s = enqueue_batch(b, b->cap, x0, V, V_safe, iter0, n_repair, b->iter_dev);
        if (s == SMPPI_OK) {
            batch_iter_inc<<<1, 1, 0, b->cap>>>(b->iter_dev);
        }
        cudaError_t e = cudaStreamEndCapture(b->cap, &g);
        if (s != SMPPI_OK) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        BCU(b, e);
        e = cudaGraphInstantiate(&b->gexec, g, 0);
        cudaGraphDestroy(g);
        BCU(b, e);
        b->graph_key = key;
    }
    BCU(b, cudaMemsetAsync(b->iter_dev, 0, sizeof(uint32_t), b->st));
    for (int i = 0; i < n_updates; ++i) BCU(b, cudaGraphLaunch(b->gexec, b->st));
    return SMPPI_OK;
}

smppi_status smppi_batch_sync_status(smppi_batch* b, uint32_t* bits_out) {
    if (!b) return bfail(nullptr, SMPPI_ERR_ARG, "batch is NULL");
    unsigned bits = 0;
    BCU(b, cudaStreamSynchronize(b->st));
    BCU(b, cudaMemcpy(&bits, b->status, sizeof(unsigned), cudaMemcpyDeviceToHost));
    BCU(b, cudaMemset(b->status, 0, sizeof(unsigned)));
    // a block that gave up on a wait left its problems' completion counters
    // behind: clear them so that the next launch starts from a clean queue
    if (bits & SMPPI_DEV_TIMEOUT) BCU(b, cudaMemset(b->done, 0, sizeof(unsigned) * b->B));
    if (bits_out) *bits_out = bits;
    if (bits & SMPPI_DEV_NUMERIC) return bfail(b, SMPPI_ERR_NUMERIC, "NaN/Inf met on the device");
    if (bits & SMPPI_DEV_TIMEOUT) return bfail(b, SMPPI_ERR_TIMEOUT, "a device wait gave up");
    if (bits & SMPPI_DEV_STALLED) return bfail(b, SMPPI_ERR_STALLED, "repair line search stalled");
    return SMPPI_OK;
}

smppi_status smppi_batch_monitor(smppi_batch* b, uint32_t* viol_out, uint32_t* outside_out,
                                 int reset) {
    if (!b) return bfail(nullptr, SMPPI_ERR_ARG, "batch is NULL");
    BCU(b, cudaStreamSynchronize(b->st));
    if (viol_out)
        BCU(b, cudaMemcpy(viol_out, b->viol, sizeof(unsigned) * b->B, cudaMemcpyDeviceToHost));
    if (outside_out)
        BCU(b, cudaMemcpy(outside_out, b->outside, sizeof(unsigned) * b->B,
                          cudaMemcpyDeviceToHost));
    if (reset) {
        BCU(b, cudaMemset(b->viol, 0, sizeof(unsigned) * b->B));
        BCU(b, cudaMemset(b->outside, 0, sizeof(unsigned) * b->B));
    }
    return SMPPI_OK;
}

smppi_status smppi_batch_config(const smppi_batch* b, int* block_rollouts, int* grid) {
    if (!b) return bfail(nullptr, SMPPI_ERR_ARG, "batch is NULL");
    if (block_rollouts) *block_rollouts = b->RB;
    if (grid) *grid = b->grid;
    return SMPPI_OK;
}

}  // extern "C"
