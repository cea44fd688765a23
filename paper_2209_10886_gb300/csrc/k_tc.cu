// Multi-RHS subdomain solves on the tensor cores (complex64 factors, TF32 inputs,
// FP32 accumulation): the batched forward/back block solves of the stored
// block-tridiagonal factorisation (Section 5, the local problems of Eq. subPbm)
// for many right-hand sides at once.  With NR right-hand sides every step
//     forward   y_r = X_r (b_r + y_{r-1}),      backward  u_r = y_r + X_r u_{r+1}
// is an (mx x mx) x (mx x NR) complex product, a dense contraction.
//
// Operands.  A complex product is two real MMAs per K-step with M = 128 output
// nodes, N = 2 NR, K = 8 (kind::tf32):
//     [Re D | Im D] = Xr [Br | Bi] + Xi [-Bi | Br]
// With SPLIT = 3 every operand is the sum of two TF32 numbers, hi = tf32(x) and
// lo = tf32(x - hi), and each real product takes three MMAs, hi*hi + hi*lo +
// lo*hi (the lo*lo term is below FP32 roundoff): FP32-level accuracy from the
// TF32 pipe.  SPLIT = 1 uses hi alone.
// The factors are re-laid out once (tc_layout_kernel) into planes of real and
// imaginary parts (hi, and lo for SPLIT = 3) in the tensor cores' no-swizzle
// K-major core-matrix layout, cut into 32 KB chunks of K; one bulk copy lands a
// chunk in shared memory ready for the MMA descriptors.  The right-hand-side
// block is the K-major B operand [-Bi | Br | Bi] (K = node index, N = 3 NR) in
// shared memory, written by the epilogue threads (a 4 x 4 shuffle transpose per
// group of four nodes, then 16-byte stores), so the two windows [Br | Bi] and
// [-Bi | Br] are both contiguous.  The accumulator D (128 lanes x 2 NR columns
// per 128-node tile) is in tensor memory.
// Descriptors (no swizzle, K-major): the leading byte offset is the distance of
// core matrices adjacent along K, the stride byte offset that of core matrices
// adjacent along M (A) or N (B).
//
// Roles.  Warps 0..15: epilogue; warp w owns the 32 nodes 32 (w mod 4MT) + lane
// of the current grid row (the TMEM lanes of its quarter, tile (w mod 4MT) / 4)
// and one of 4/MT groups of the right-hand sides.  Warp 16: producer (one thread
// issues the bulk copies into a ring of chunk slots); warp 17: one thread issues
// the MMAs and commits them to mbarriers.  Per step the epilogue waits for the
// accumulator, forms the next operand (b_{r+1} + y_r, or y_r + X_r u_{r+1} on the
// way back) and signals the MMA thread; its global operands (y_r, the source,
// the interface data) are loaded one chunk of 4 RHS ahead, the first chunk while
// the MMAs run.  The interface data G/(1-beta) of all boundary nodes are gathered
// once per launch into a scratch array, and the outgoing data are formed after
// the sweep from the boundary values kept in a second one, by all threads.  All
// waits are bounded: on expiry the kernel records HELM_ERR_TIMEOUT, stops issuing
// work, waits (bounded) for its own copies and MMAs and frees its tensor memory.
#include "helm_internal.cuh"

#include <algorithm>

namespace {

constexpr long long TC_WAIT_LIMIT = 2000000000LL;  // cycles (~1 s)
constexpr int TC_MAXSLOTS = 8;
constexpr int TC_CHUNK_BYTES = 32768;              // one K-chunk: real plane + imaginary plane
constexpr int TC_EPI_WARPS = 16;                   // epilogue warps (4 MT per node set x RHS groups)

__device__ __forceinline__ unsigned sm_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(unsigned long long* b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(sm_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_arrive(unsigned long long* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(sm_addr(b)) : "memory");
}
__device__ __forceinline__ void bar_expect_tx(unsigned long long* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(sm_addr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool bar_try(unsigned long long* b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(sm_addr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool bar_wait(unsigned long long* b, unsigned parity, long long limit) {
    if (bar_try(b, parity)) return true;
    const long long t0 = clock64();
    while (!bar_try(b, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    if (!HELM_CHK(src, bytes)) return;                  // checking build: the wait then gives up
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(sm_addr(dst)),
        "l"(src), "r"(bytes), "r"(sm_addr(bar))
        : "memory");
}

// shared-memory matrix descriptor, no swizzle: start, leading and stride byte offsets (>> 4),
// bits 46-48 = 0b001
__device__ __forceinline__ unsigned long long smem_desc(unsigned addr, unsigned lbo, unsigned sbo) {
    return (unsigned long long)((addr >> 4) & 0x3FFFu) | ((unsigned long long)((lbo >> 4) & 0x3FFFu) << 16) |
           ((unsigned long long)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// instruction descriptor of kind::tf32: D f32, A and B tf32, both K-major, N, M = 128
__host__ __device__ constexpr unsigned tf32_idesc(int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(n >> 3) << 17) | ((128u >> 4) << 24);
}
__device__ __forceinline__ void mma_tf32(unsigned dtmem, unsigned long long adesc, unsigned long long bdesc,
                                         unsigned idesc, int accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(unsigned long long* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(sm_addr(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
// 8 consecutive 32-bit columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld8(unsigned addr, float* v) {
    unsigned r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(addr));
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}
// 4 consecutive 32-bit columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld4(unsigned addr, float* v) {
    unsigned r[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = __uint_as_float(r[j]);
}
// binary32 -> binary64 widening of a normal number by its bit fields (sign, exponent
// rebiased by 1023 - 127, mantissa shifted by 52 - 23): integer instructions instead of
// a conversion on the FP64 pipe; zero, subnormals, infinities and NaN take the conversion
__device__ __forceinline__ double widen(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xFFu;
    if (e == 0u || e == 0xFFu) return (double)f;
    const unsigned long long d = ((unsigned long long)(u & 0x80000000u) << 32) |
                                 ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)d);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }
__device__ __forceinline__ float tf32_round(float x) {
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}
__device__ __forceinline__ void st_shared_v4(unsigned addr, float a, float b, float c, float d) {
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};\n" ::"r"(addr), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}

}  // namespace

// ----------------------------------------------------------------- layout
// XT of one subdomain: my steps x nch chunks of 32 KB; chunk c holds K columns
// [c*KC, c*KC + KC) of all 128*MT rows as planes (real hi, imaginary hi, and for
// SPLIT = 3 real lo, imaginary lo; KC = 32 / (MT * SPLIT') with SPLIT' = 1 or 2
// planes per part), each of core matrices 8 rows x 4 columns:
//     float index in a plane = ((kl / 4) * 16 MT + i / 8) * 32 + (i % 8) * 4 + kl % 4
// Rows i >= mx and columns j >= mx are zero; values are rounded to TF32.
__host__ __device__ inline int tc_kc(int MT, int split) { return (split == 3 ? 16 : 32) / MT; }

__global__ void tc_layout_kernel(const SubDev* subtab, int nsub, int split, const float2* X, float* XT) {
    const int s = blockIdx.y;
    if (s >= nsub) return;
    const SubDev sd = subtab[s];
    const int MT = sd.tcmt;
    if (MT < 1 || MT > 2) return;
    const int KC = tc_kc(MT, split);
    const int nch = (sd.mx + KC - 1) / KC;
    const long long per_step = (long long)nch * (TC_CHUNK_BYTES / 4);
    const long long total = (long long)sd.my * per_step;
    const int plane = 128 * MT * KC;                       // floats per plane
    for (long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x; f < total;
         f += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(f / per_step);
        const long long g = f - (long long)r * per_step;
        const int np = split == 3 ? 4 : 2;
        const int c = (int)(g / (np * plane));
        const int h = (int)(g - (long long)c * np * plane);
        const int p = h / plane;                           // 0 real hi, 1 imaginary hi, 2 real lo, 3 imaginary lo
        const int q = h - p * plane;
        const int core = q >> 5, w = q & 31;
        const int ck = core / (16 * MT), cm = core - ck * 16 * MT;
        const int i = cm * 8 + (w >> 2);
        const int j = c * KC + ck * 4 + (w & 3);
        float v = 0.f;
        if (i < sd.mx && j < sd.mx) {
            const long long e = j < sd.w0 ? (long long)i * sd.ld0 + j
                                          : (long long)sd.mx * sd.ld0 + (long long)i * sd.ld1 + (j - sd.w0);
            const float2 x = HLD(X + sd.xoff + (long long)r * sd.mx * (sd.ld0 + sd.ld1) + e);
            const float xv = (p & 1) ? x.y : x.x;
            const float hi = tf32_round(xv);
            v = p < 2 ? hi : tf32_round(xv - hi);
        }
        HST(XT + sd.xtoff + f, v);
    }
}

namespace {

// ------------------------------------------------------------- stage kernel
template <int MT, int NR, bool BASIS, int SPLIT>
__global__ void __launch_bounds__(32 * (TC_EPI_WARPS + 2), 1)
    tc_stage_kernel(StageArgs<float> a, const float* __restrict__ XT, int nslots) {
    using T = float2;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long full_bar[TC_MAXSLOTS], empty_bar[TC_MAXSLOTS], b_bar, d_bar, fin_bar;
    __shared__ unsigned tmem_base;
    __shared__ int abort_flag;
    __shared__ float zsc_s[NR];                             // per-RHS output scales

    constexpr int NEPI = 32 * TC_EPI_WARPS;                 // epilogue threads
    constexpr int NW = 4 * MT;                              // warps per set of 128*MT nodes
    constexpr int RG = TC_EPI_WARPS / NW;                   // RHS groups: each epilogue warp takes NR/RG RHS
    constexpr int RPT = NR / RG;                            // RHS per epilogue thread
    static_assert(RPT % 4 == 0, "RHS per epilogue thread must be a multiple of 4");
    constexpr int CH = RPT >= 8 ? 8 : 4;                    // RHS per chunk of the epilogue
    constexpr int KC = (SPLIT == 3 ? 16 : 32) / MT;         // K columns per chunk
    constexpr unsigned PLANE = 128u * MT * KC * 4u;         // bytes of one plane of a chunk
    constexpr unsigned BLO = 32u * MT * (48u * NR + 64u);  // offset of the lo operand (SPLIT = 3)
    constexpr int NCOLS = 2 * NR * MT;                      // accumulator columns
    constexpr int TCOLS = NCOLS <= 32 ? 32 : NCOLS <= 64 ? 64 : NCOLS <= 128 ? 128 : NCOLS <= 256 ? 256 : 512;
    // B operand: core matrix (n / 8, node / 4) at (node / 4) * KSTRIDE_B + (n / 8) * 128; the
    // extra 64 bytes put consecutive node groups in opposite halves of the banks
    constexpr unsigned KSTRIDE_B = 48u * NR + 64u;
    constexpr unsigned KSTRIDE_A = 2048u * MT;              // K-adjacent core matrices of A
    constexpr unsigned IDESC = tf32_idesc(2 * NR);

    const int s = HLD(a.subs + blockIdx.x);
    const SubDev sd = HLD(a.subtab + s);
    const int mx = sd.mx, my = sd.my;
    const int rhs0 = blockIdx.y * NR;
    const int e0 = BASIS ? a.col0 + rhs0 : 0;
    if (BASIS && e0 >= sd.Lb) return;                       // uniform over the CTA
    const int nr = BASIS ? min(NR, sd.Lb - e0) : min(NR, a.nrhs - rhs0);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nch = (mx + KC - 1) / KC;
    const int nsteps = 2 * my - 1;
    const long long N = (long long)a.nx * a.ny;
    const int L = 2 * (mx + my);                            // boundary slots W[my] E[my] S[mx] N[mx]
    const bool has_gin = !BASIS && (a.gin0 || a.gin1);

    unsigned char* ring = smem_raw;
    unsigned char* bop = smem_raw + (size_t)nslots * TC_CHUNK_BYTES;   // [-Bi | Br | Bi] (hi, then lo)
    const unsigned ring_s = sm_addr(ring), bop_s = sm_addr(bop);

    if (tid == 0) {
        for (int i = 0; i < nslots; ++i) {
            bar_init(&full_bar[i], 1);
            bar_init(&empty_bar[i], 1);
        }
        bar_init(&b_bar, NEPI);
        bar_init(&d_bar, 1);
        bar_init(&fin_bar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    for (int k = tid; k < NR; k += blockDim.x) zsc_s[k] = (!BASIS && a.zscale && k < nr) ? (float)HLD(a.zscale + rhs0 + k) : 1.f;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(sm_addr(&tmem_base)),
                     "r"(TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }

    // the four sides with compile-time indices (no local-memory arrays)
    const int tinW = sd.tin[SW], tinE = sd.tin[SE], tinS = sd.tin[SS], tinN = sd.tin[SN];
    const int boW = sd.bo[SW], boE = sd.bo[SE], boS = sd.bo[SS], boN = sd.bo[SN];
    auto gin = [&](int k, long long idx) -> T {
        T g = a.gin0 ? HLD(a.gin0 + (long long)(rhs0 + k) * a.ntrace + idx) : czero<T>();
        if (a.gin1) g = cadd(g, HLD(a.gin1 + (long long)(rhs0 + k) * a.ntrace + idx));
        return g;
    };
    // interface part of the right-hand side at boundary node (r, cc) for RHS k: the
    // incoming data G/(1-beta) of every side through the node, or the unit datum (basis)
    auto bside = [&](int tin, int bo, int pt, int k, T b) -> T {
        if (BASIS) {
            if (bo >= 0 && bo + pt == e0 + k) b = cadd(b, mk(1.f, 0.f));
        } else if (tin >= 0 && has_gin) {
            const long long ti = tin + pt;
            b = cadd(b, cmul(gin(k, ti), HLD(a.tc + ti).cin));
        }
        return b;
    };
    auto bnode = [&](int r, int cc, int k) -> T {
        T b = czero<T>();
        if (cc == 0) b = bside(tinW, boW, r, k, b);
        if (cc == mx - 1) b = bside(tinE, boE, r, k, b);
        if (r == 0) b = bside(tinS, boS, cc, k, b);
        if (r == my - 1) b = bside(tinN, boN, cc, k, b);
        return b;
    };
    // the one boundary slot that carries node (r, cc)'s interface data (its W or E entry
    // on the edge columns, else its S or N entry), -1 for interior nodes
    auto node_slot = [&](int r, int cc) -> int {
        return cc == 0 ? r : cc == mx - 1 ? my + r : r == 0 ? 2 * my + cc : r == my - 1 ? 2 * my + mx + cc : -1;
    };
    T* escr = has_gin ? a.escr + (long long)rhs0 * a.estride + sd.eoff : nullptr;   // [k * estride + slot]
    if (has_gin) {
        // incoming data of every boundary node and RHS, once per launch (all threads, loads in parallel)
        for (int idx = tid; idx < nr * L; idx += blockDim.x) {
            const int k = idx / L, e = idx - k * L;
            const int r = e < my ? e : e < 2 * my ? e - my : e < 2 * my + mx ? 0 : my - 1;
            const int cc = e < my ? 0 : e < 2 * my ? mx - 1 : e < 2 * my + mx ? e - 2 * my : e - 2 * my - mx;
            if (node_slot(r, cc) != e) continue;            // a corner's S/N entry, or E when mx = 1
            HST(escr + (long long)k * a.estride + e, bnode(r, cc, k));
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = tmem_base;

    auto fail = [&]() {
        abort_flag = 1;
        if (a.err) atomicExch(a.err, (int)HELM_ERR_TIMEOUT);
    };
    auto aborted = [&]() { return *((volatile int*)&abort_flag) != 0; };

    if (warp < TC_EPI_WARPS) {
        // ------------------------------------------------------------ epilogue
        // warp w: nodes 32 (w % NW) + lane (TMEM lanes of its quarter), RHS [kb, kb + RPT)
        const int nw = warp % NW;
        const int c = 32 * nw + lane;
        const int tile = nw >> 2;
        const int kb = (warp / NW) * RPT;
        const unsigned dcol = tmem + ((unsigned)(32 * (warp & 3)) << 16) + (unsigned)(tile * 2 * NR);
        const bool live = c < mx;
        const unsigned bgrp = bop_s + (unsigned)(c >> 2) * KSTRIDE_B;      // K core matrix of nodes 4(c/4) ..
        T* yw = a.yws + sd.yoff;
        T* uscr = (!BASIS && a.mask) ? a.uscr + (long long)rhs0 * a.estride + sd.eoff : nullptr;
        const bool edge_col = c == 0 || c == mx - 1;
        // u is the solution at boundary node (r, c) for RHS k: K entries (basis) or the
        // value kept for the outgoing data of every interface side through the node
        auto finish_edge = [&](int r, int k, T u) {
            auto one = [&](int tin, int bo, int e, int pt) {
                if (BASIS) {
                    if (bo >= 0) HST(a.K + sd.koff + (long long)(e0 + k) * sd.Lb + bo + pt, u);
                } else if (uscr && tin >= 0) {
                    HST(uscr + (long long)k * a.estride + e, u);
                }
            };
            if (c == 0) one(tinW, boW, r, r);
            if (c == mx - 1) one(tinE, boE, my + r, r);
            if (r == 0) one(tinS, boS, 2 * my + c, c);
            if (r == my - 1) one(tinN, boN, 2 * my + mx + c, c);
        };
        // write the operand entries of RHS k0 .. k0+3 (v[j] = value of RHS k0 + j at this
        // node): a 4 x 4 transpose within each group of four lanes leaves lane j of the
        // group with RHS k0 + j at the group's four nodes, one 16-byte row of a core matrix
        auto put4 = [&](int k0, const T* v) {
            const int j = lane & 3, gb = lane & ~3;
            float wr[4], wi[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int sj = (j - q) & 3, i = (j + q) & 3;
                const float sr = sj == 0 ? v[0].x : sj == 1 ? v[1].x : sj == 2 ? v[2].x : v[3].x;
                const float si = sj == 0 ? v[0].y : sj == 1 ? v[1].y : sj == 2 ? v[2].y : v[3].y;
                const float rr = __shfl_sync(0xffffffffu, sr, gb | i);
                const float ri = __shfl_sync(0xffffffffu, si, gb | i);
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    if (t == i) { wr[t] = rr; wi[t] = ri; }
                }
            }
            const int n = k0 + j;
            auto row = [&](int nn) { return bgrp + (unsigned)(nn >> 3) * 128u + (unsigned)(nn & 7) * 16u; };
            float hr[4], hi[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) { hr[t] = tf32_round(wr[t]); hi[t] = tf32_round(wi[t]); }
            st_shared_v4(row(n), -hi[0], -hi[1], -hi[2], -hi[3]);
            st_shared_v4(row(NR + n), hr[0], hr[1], hr[2], hr[3]);
            st_shared_v4(row(2 * NR + n), hi[0], hi[1], hi[2], hi[3]);
            if (SPLIT == 3) {
                float lr[4], li[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) { lr[t] = tf32_round(wr[t] - hr[t]); li[t] = tf32_round(wi[t] - hi[t]); }
                st_shared_v4(BLO + row(n), -li[0], -li[1], -li[2], -li[3]);
                st_shared_v4(BLO + row(NR + n), lr[0], lr[1], lr[2], lr[3]);
                st_shared_v4(BLO + row(2 * NR + n), li[0], li[1], li[2], li[3]);
            }
        };
        // operand of step 0: b_1
        for (int k0 = kb; k0 < kb + RPT; k0 += 4) {
            T v[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int k = k0 + j;
                T b = czero<T>();
                if (live && k < nr) {
                    const int sl = node_slot(0, c);
                    if (sl >= 0) b = has_gin ? HLD(escr + (long long)k * a.estride + sl) : bnode(0, c, k);
                    if (!BASIS && a.src) b = cadd(b, HLD(a.r64 + (long long)(rhs0 + k) * N + (long long)sd.y0 * a.nx + sd.x0 + c));
                }
                v[j] = b;
            }
            put4(k0, v);
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        tc_fence_before();
        bar_arrive(&b_bar);
        const long long ws = a.wstride;
        for (int step = 0; step < nsteps; ++step) {
            const bool fwd = step < my;
            const int r = fwd ? step : 2 * my - 2 - step;
            // what this step does at this node, decided once per step:
            //   mid (forward, r < my-1): store y_r, next operand b_{r+1} + y_r
            //   otherwise the solution of row r is final: u = y_my (r = my-1) or y_r + X_r u_{r+1}
            const bool mid = fwd && r < my - 1;
            const bool ok = live && !aborted();
            T* yrow = yw + (long long)rhs0 * ws + (long long)r * mx + c;          // y_r of RHS rhs0
            const T* srow = (!BASIS && a.src && mid && ok)
                                ? a.r64 + (long long)rhs0 * N + (long long)(sd.y0 + r + 1) * a.nx + sd.x0 + c
                                : nullptr;
            double2* zrow = (!BASIS && a.z && !mid && ok)
                                ? a.z + (long long)rhs0 * N + (long long)(sd.y0 + r) * a.nx + sd.x0 + c
                                : nullptr;
            const int nslot = mid ? node_slot(r + 1, c) : -1;                     // interface data in row r+1
            const T* erow = (has_gin && ok && nslot >= 0) ? escr + nslot : nullptr;
            const bool bunit = BASIS && mid && nslot >= 0;
            const bool fedge = !mid && (edge_col || r == 0 || r == my - 1);
            const bool loady = !fwd && ok;
            // global operands of one chunk of CH RHS, loaded a chunk ahead (the first one
            // before the accumulator wait, under the MMAs): pv = y_r on the way back or the
            // source of row r+1 on the way forward, ev = the interface data of row r+1
            auto prefetch = [&](int k0, T* pv, T* ev) {
#pragma unroll
                for (int j = 0; j < CH; ++j) {
                    const int k = k0 + j;
                    pv[j] = czero<T>();
                    ev[j] = czero<T>();
                    if (k < nr) {
                        if (loady) pv[j] = yrow[(long long)k * ws];
                        else if (srow) pv[j] = srow[(long long)k * N];
                        if (erow) ev[j] = HLD(erow + (long long)k * a.estride);
                    }
                }
            };
            T pv[CH], ev[CH];
            prefetch(kb, pv, ev);
            if (!bar_wait(&d_bar, (unsigned)(step & 1), aborted() ? 0 : TC_WAIT_LIMIT)) fail();
            tc_fence_after();
            const bool last = step == nsteps - 1;
#pragma unroll 1
            for (int k0 = kb; k0 < kb + RPT; k0 += CH) {
                T pn[CH], en[CH];
                if (k0 + CH < kb + RPT) prefetch(k0 + CH, pn, en);
                float dr[CH], di[CH];
                if (CH == 8) {
                    tmem_ld8(dcol + (unsigned)k0, dr);
                    tmem_ld8(dcol + (unsigned)(NR + k0), di);
                } else {
                    tmem_ld4(dcol + (unsigned)k0, dr);
                    tmem_ld4(dcol + (unsigned)(NR + k0), di);
                }
                tmem_wait_ld();
                T nv[CH];
                if (ok) {
                    T* yk = yrow + (long long)k0 * ws;
#pragma unroll
                    for (int j = 0; j < CH; ++j, yk += ws) {
                        const int k = k0 + j;
                        const T sum = mk(dr[j], di[j]);
                        T v = czero<T>();
                        if (k < nr) {
                            if (mid) {
                                *yk = sum;                                        // y_r
                                v = cadd(sum, pv[j]);                             // + source of row r+1
                                if (erow) v = cadd(v, ev[j]);                     // + interface data
                                if (bunit) v = cadd(v, bnode(r + 1, c, k));       // + unit datum (basis)
                            } else {
                                v = fwd ? sum : cadd(pv[j], sum);                 // u_my = y_my, u_r = y_r + X_r u_{r+1}
                                if (zrow) {
                                    const float sc = zsc_s[k];
                                    zrow[(long long)k * N] = make_double2(widen(v.x * sc), widen(v.y * sc));
                                }
                                if (fedge) finish_edge(r, k, v);
                            }
                        }
                        nv[j] = v;
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < CH; ++j) nv[j] = czero<T>();
                }
                if (!last) {
#pragma unroll
                    for (int j = 0; j < CH; j += 4) put4(k0 + j, nv + j);
                }
#pragma unroll
                for (int j = 0; j < CH; ++j) { pv[j] = pn[j]; ev[j] = en[j]; }
            }
            if (!last) {
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                tc_fence_before();
                bar_arrive(&b_bar);
            }
        }
    } else if (warp == TC_EPI_WARPS) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            const float* Xs = XT + sd.xtoff;
            const long long chunk_f = TC_CHUNK_BYTES / 4;
            int slot = 0, issued = 0;
            unsigned ph = 0;
            for (int step = 0; step < nsteps && !aborted(); ++step) {
                const int r = step < my ? step : 2 * my - 2 - step;
                for (int ch = 0; ch < nch; ++ch) {
                    if (aborted()) break;
                    if (issued >= nslots && !bar_wait(&empty_bar[slot], ph ^ 1u, TC_WAIT_LIMIT)) {
                        fail();
                        break;
                    }
                    bar_expect_tx(&full_bar[slot], TC_CHUNK_BYTES);
                    bulk_load(ring + (size_t)slot * TC_CHUNK_BYTES, Xs + ((long long)r * nch + ch) * chunk_f,
                              TC_CHUNK_BYTES, &full_bar[slot]);
                    ++issued;
                    if (++slot == nslots) { slot = 0; ph ^= 1u; }
                }
            }
            if (aborted()) {
                for (int t = max(0, issued - nslots); t < issued; ++t)
                    bar_wait(&full_bar[t % nslots], (unsigned)((t / nslots) & 1), TC_WAIT_LIMIT);
            } else {
                // the last releases of every slot have landed before the CTA leaves
                for (int t = max(0, issued - nslots); t < issued; ++t)
                    if (!bar_wait(&empty_bar[t % nslots], (unsigned)((t / nslots) & 1), TC_WAIT_LIMIT)) fail();
            }
        }
    } else {
        // ------------------------------------------------------------ MMA issue
        if (lane == 0) {
            int slot = 0;
            unsigned ph = 0;
            bool any = false;
            for (int step = 0; step < nsteps; ++step) {
                if (!bar_wait(&b_bar, (unsigned)(step & 1), aborted() ? 0 : TC_WAIT_LIMIT)) fail();
                if (aborted()) break;
                tc_fence_after();
                for (int ch = 0; ch < nch; ++ch) {
                    if (!bar_wait(&full_bar[slot], ph, TC_WAIT_LIMIT)) { fail(); break; }
                    tc_fence_after();
                    const unsigned abase = ring_s + (unsigned)slot * TC_CHUNK_BYTES;
#pragma unroll
                    for (int kk = 0; kk < KC / 8; ++kk) {
                        const int kc = (ch * KC + kk * 8) >> 2;          // first K core matrix of the B operand
                        const unsigned bb = bop_s + (unsigned)kc * KSTRIDE_B;
                        const unsigned long long b1 = smem_desc(bb + (unsigned)(NR / 8) * 128u, KSTRIDE_B, 128u);
                        const unsigned long long b2 = smem_desc(bb, KSTRIDE_B, 128u);
#pragma unroll
                        for (int t = 0; t < MT; ++t) {
                            const unsigned ar = abase + (unsigned)kk * 2u * KSTRIDE_A + (unsigned)t * 2048u;
                            const unsigned long long dre = smem_desc(ar, KSTRIDE_A, 128u);
                            const unsigned long long dim = smem_desc(ar + PLANE, KSTRIDE_A, 128u);
                            const unsigned dt = tmem + (unsigned)(t * 2 * NR);
                            mma_tf32(dt, dre, b1, IDESC, (ch > 0 || kk > 0) ? 1 : 0);
                            mma_tf32(dt, dim, b2, IDESC, 1);
                            if (SPLIT == 3) {
                                const unsigned long long b1l = smem_desc(BLO + bb + (unsigned)(NR / 8) * 128u, KSTRIDE_B, 128u);
                                const unsigned long long b2l = smem_desc(BLO + bb, KSTRIDE_B, 128u);
                                const unsigned long long drel = smem_desc(ar + 2u * PLANE, KSTRIDE_A, 128u);
                                const unsigned long long diml = smem_desc(ar + 3u * PLANE, KSTRIDE_A, 128u);
                                mma_tf32(dt, dre, b1l, IDESC, 1);      // hi * lo
                                mma_tf32(dt, dim, b2l, IDESC, 1);
                                mma_tf32(dt, drel, b1, IDESC, 1);      // lo * hi
                                mma_tf32(dt, diml, b2, IDESC, 1);
                            }
                        }
                    }
                    mma_commit(&empty_bar[slot]);                        // slot free once these complete
                    any = true;
                    if (++slot == nslots) { slot = 0; ph ^= 1u; }
                }
                if (aborted()) break;
                mma_commit(&d_bar);                                      // accumulator of this step ready
            }
            if (any) {
                // every MMA this thread issued has completed before tensor memory is freed
                mma_commit(&fin_bar);
                bar_wait(&fin_bar, 0u, TC_WAIT_LIMIT);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TCOLS) : "memory");
    }
    // outgoing data G_out = ca G_in + cb u_p toward the masked sides, all threads at once
    // (the boundary values u_p were kept during the sweep)
    if (!BASIS && a.mask && !abort_flag) {
        const T* uscr = a.uscr + (long long)rhs0 * a.estride + sd.eoff;
        const int toutW = sd.tout[SW], toutE = sd.tout[SE], toutS = sd.tout[SS], toutN = sd.tout[SN];
        for (int idx = tid; idx < nr * L; idx += blockDim.x) {
            const int k = idx / L, e = idx - k * L;
            const int side = e < my ? SW : e < 2 * my ? SE : e < 2 * my + mx ? SS : SN;
            const int pt = e < my ? e : e < 2 * my ? e - my : e < 2 * my + mx ? e - 2 * my : e - 2 * my - mx;
            const int tin = side == SW ? tinW : side == SE ? tinE : side == SS ? tinS : tinN;
            const int tout = side == SW ? toutW : side == SE ? toutE : side == SS ? toutS : toutN;
            if (!(a.mask & (1 << side)) || tin < 0) continue;
            const long long in = tin + pt, out = tout + pt;
            const TraceCoef<T> cf = HLD(a.tc + in);
            T g = cfma(cf.cb, HLD(uscr + (long long)k * a.estride + e), cmul(cf.ca, gin(k, in)));
            const long long o = (long long)(rhs0 + k) * a.ntrace + out;
            if (a.base) g = cadd(g, HLD(a.base + o));
            if (a.sub) g = csub(g, HLD(a.sub + o));
            HST(a.dst + o, g);
            if (a.dst2) HST(a.dst2 + o, g);
        }
    }
}

template <int MT, int NR, int SPLIT>
size_t tc_smem(int nslots) {
    return (size_t)nslots * TC_CHUNK_BYTES + (size_t)32 * MT * (48 * NR + 64) * (SPLIT == 3 ? 2 : 1);
}

template <int MT, int NR, bool BASIS, int SPLIT>
cudaError_t tc_launch(const StageArgs<float>& a, const float* XT, int nunits, int ny_blocks, cudaStream_t st) {
    // dynamic shared memory: at most 227 KB per block less the kernel's static shared memory
    cudaFuncAttributes fa{};
    cudaError_t e0 = cudaFuncGetAttributes(&fa, tc_stage_kernel<MT, NR, BASIS, SPLIT>);
    if (e0 != cudaSuccess) return e0;
    const size_t budget = 227 * 1024 - fa.sharedSizeBytes - 256;
    int nslots = TC_MAXSLOTS;
    while (nslots > 2 && tc_smem<MT, NR, SPLIT>(nslots) > budget) --nslots;
    if (tc_smem<MT, NR, SPLIT>(nslots) > budget) return cudaErrorInvalidValue;
    const size_t smem = tc_smem<MT, NR, SPLIT>(nslots);
    cudaError_t e = cudaFuncSetAttribute(tc_stage_kernel<MT, NR, BASIS, SPLIT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    count_launch();
    tc_stage_kernel<MT, NR, BASIS, SPLIT><<<dim3(nunits, ny_blocks), 32 * (TC_EPI_WARPS + 2), smem, st>>>(a, XT, nslots);
    return cudaGetLastError();
}

// ------------------------------------------------- interface stages, many RHS
// One interface stage with NB right-hand sides per CTA as a complex GEMM on the tensor
// cores: for the output rows (points of the masked sides) of one subdomain,
//     D = K_rows (cin * G)       (K: Lb boundary points wide, G: incoming data, NB RHS)
// then G_out = cb D + ca G_in + base - sub per row and RHS, as the CUDA-core form of the
// stage computes it.  A CTA takes 128 rows (one M tile) and NB RHS, and walks the
// boundary points in chunks of KC = 16: its four warps load the next chunk's K rows
// (coalesced: 16 lanes per row) and incoming data into registers, write the current one
// into a double-buffered pair of operands (A: real and imaginary planes of K; B:
// [-Gi | Gr | Gi]; each split into TF32 hi and lo for SPLIT = 3; no-swizzle K-major
// core-matrix layouts as in the stage kernel, A's K groups padded by 16 bytes against
// bank conflicts) and one thread issues the chunk's MMAs, committed to the buffer's
// mbarrier, while the warps move on.  The accumulator [Re D | Im D] (128 lanes
// x 2 NB columns) is in tensor memory; warp w reads lanes 32w.. for the epilogue.  With
// S > 1 a tile's chunks are split over S CTAs: each stores its partial sums, and the last
// to arrive (one counter per tile, reset by that CTA) adds the S partials in split order
// and finishes the tile, so the sums do not depend on which CTA ends last.  Waits are
// bounded: on expiry the CTA records HELM_ERR_TIMEOUT, issues nothing more, waits
// (bounded) for its MMAs and frees its tensor memory.
template <int NB, int SPLIT>
__global__ void __launch_bounds__(128, 1) tc_iface_kernel(IfaceArgs<float> a, int S) {
    using T = float2;
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long mma_bar[2], fin_bar;
    __shared__ unsigned tmem_base;
    __shared__ int abort_flag;

    constexpr int KC = 16;                                  // boundary points per chunk
    // A: K-adjacent core matrices 2048 + 16 bytes apart, so that the 16 points of a row
    // written by 16 lanes fall in 16 different banks
    constexpr unsigned KSA = 2064u;
    constexpr unsigned PLANE = (KC / 4) * KSA;              // one plane of A
    constexpr unsigned ABYTES = (SPLIT == 3 ? 4u : 2u) * PLANE;
    constexpr unsigned KSB = 48u * NB;                      // K-adjacent core matrices of B
    constexpr unsigned BPART = (KC / 4) * KSB;              // B hi (and B lo after it)
    constexpr unsigned BBYTES = (SPLIT == 3 ? 2u : 1u) * BPART;
    constexpr int NCOLS = 2 * NB;                           // [Re D | Im D]
    constexpr int TCOLS = NCOLS <= 32 ? 32 : NCOLS <= 64 ? 64 : 128;
    constexpr unsigned IDESC = tf32_idesc(2 * NB);
    constexpr int PPT = (4 * NB + 127) / 128;               // (point quad, RHS) pairs per thread


    const int rhs0 = blockIdx.x * NB;
    const int nr = min(NB, a.nrhs - rhs0);
    const int row0 = blockIdx.y * 128;
    const int slot = blockIdx.z / S, split = blockIdx.z - slot * S;   // S CTAs share one output tile
    const SubDev sd = HLD(a.subtab + HLD(a.subs + slot));
    const int Lb = sd.Lb;
    const int bo[4] = {sd.bo[0], sd.bo[1], sd.bo[2], sd.bo[3]};
    const int tin[4] = {sd.tin[0], sd.tin[1], sd.tin[2], sd.tin[3]};
    auto sel = [&](const int (&v)[4], int q) { return q == 0 ? v[0] : q == 1 ? v[1] : q == 2 ? v[2] : v[3]; };
    auto len = [&](int q) { return q < 2 ? sd.my : sd.mx; };
    auto on = [&](int q) { return ((a.mask >> q) & 1) && sel(bo, q) >= 0; };
    int rcount = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (on(q)) rcount += len(q);
    if (row0 >= rcount || nr <= 0) return;                  // uniform over the CTA
    const int tid = threadIdx.x, warp = tid >> 5;

    // this thread's output row: side srow, point pt (srow = -1 past the last row)
    int srow = -1, pt = row0 + tid;
    if (row0 + tid < rcount) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (srow < 0 && on(q)) {
                if (pt < len(q)) srow = q;
                else pt -= len(q);
            }
    }
    const bool live = srow >= 0;
    __shared__ long long rowoff[128];                       // element offset of each row of K (-1: none)
    rowoff[tid] = live ? sd.koff + (long long)(sel(bo, srow) + pt) * Lb : -1LL;
    // this CTA's chunks of boundary points: [cb0, cb1) of the tile's (Lb + KC - 1) / KC
    const int nall = (Lb + KC - 1) / KC;
    const int cb0 = (int)((long long)split * nall / S), cb1 = (int)((long long)(split + 1) * nall / S);
    const int nch = cb1 - cb0;

    if (tid == 0) {
        bar_init(&mma_bar[0], 1);
        bar_init(&mma_bar[1], 1);
        bar_init(&fin_bar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(sm_addr(&tmem_base)),
                     "r"(TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    const unsigned sbase = sm_addr(smem_raw);
    auto abuf = [&](int b) { return sbase + (unsigned)b * ABYTES; };
    auto bbuf = [&](int b) { return sbase + 2u * ABYTES + (unsigned)b * BBYTES; };
    // K of chunk c for the warp's 32 rows, coalesced: load i takes row 32 w + r_i (lanes
    // 0-15) and row 32 w + r_i + 4 (lanes 16-31), point lane % 16 of the chunk, with
    // r_i = 8 (i / 4) + i % 4
    const int lhalf = (tid & 31) >> 4, lcol = tid & 15;
    auto krow_of = [&](int i) { return 32 * warp + 8 * (i >> 2) + (i & 3) + 4 * lhalf; };
    auto load_k = [&](int c, T (&kv)[KC]) {
        const int col = (cb0 + c) * KC + lcol;
#pragma unroll
        for (int i = 0; i < KC; ++i) {
            const long long ro = rowoff[krow_of(i)];
            kv[i] = (ro >= 0 && col < Lb) ? HLD(a.K + ro + col) : make_float2(0.f, 0.f);
        }
    };
    // incoming data of the thread's (quad, RHS) pairs: quad = pair % 4, RHS = pair / 4
    auto load_g = [&](int c, T (&gv)[PPT][4], T (&cv)[PPT][4]) {
#pragma unroll
        for (int u = 0; u < PPT; ++u) {
            const int pr = tid + 128 * u;
            const int quad = pr & 3, k = pr >> 2;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int e = (cb0 + c) * KC + 4 * quad + q;
                T G = make_float2(0.f, 0.f), C = G;
                if (pr < 4 * NB && k < nr && e < Lb) {
                    int sd_ = 0;
#pragma unroll
                    for (int t = 1; t < 4; ++t)
                        if (bo[t] >= 0 && e >= bo[t]) sd_ = t;
                    const long long ti = sel(tin, sd_) + (e - sel(bo, sd_));
                    const long long o = (long long)(rhs0 + k) * a.ntrace + ti;
                    if (a.gin0) G = HLD(a.gin0 + o);
                    if (a.gin1) G = cadd(G, HLD(a.gin1 + o));
                    C = HLD(a.tc + ti).cin;
                }
                gv[u][q] = G;
                cv[u][q] = C;
            }
        }
    };
    // operands of chunk c into buffer b: A from the raw K rows (thread t: row t), B from
    // the incoming data in registers
    auto store = [&](int b, const T (&kv)[KC], const T (&gv)[PPT][4], const T (&cv)[PPT][4]) {
        // element (row, point) of a plane at (point / 4) KSA + (row / 8) 128 + (row % 8) 16 + (point % 4) 4
        const unsigned acol = abuf(b) + (unsigned)(lcol >> 2) * KSA + (unsigned)(lcol & 3) * 4u;
#pragma unroll
        for (int i = 0; i < KC; ++i) {
            const int row = krow_of(i);
            const unsigned ad = acol + (unsigned)(row >> 3) * 128u + (unsigned)(row & 7) * 16u;
            const float hr = tf32_round(kv[i].x), hi = tf32_round(kv[i].y);
            asm volatile("st.shared.f32 [%0], %1;\n" ::"r"(ad), "f"(hr) : "memory");
            asm volatile("st.shared.f32 [%0], %1;\n" ::"r"(ad + PLANE), "f"(hi) : "memory");
            if (SPLIT == 3) {
                asm volatile("st.shared.f32 [%0], %1;\n" ::"r"(ad + 2u * PLANE), "f"(tf32_round(kv[i].x - hr)) : "memory");
                asm volatile("st.shared.f32 [%0], %1;\n" ::"r"(ad + 3u * PLANE), "f"(tf32_round(kv[i].y - hi)) : "memory");
            }
        }
#pragma unroll
        for (int u = 0; u < PPT; ++u) {
            const int pr = tid + 128 * u;
            if (pr < 4 * NB) {
                const int quad = pr & 3, k = pr >> 2;
                float gr[4], gi[4], lr[4], li[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const T g = cmul(gv[u][q], cv[u][q]);
                    gr[q] = tf32_round(g.x);
                    gi[q] = tf32_round(g.y);
                    lr[q] = tf32_round(g.x - gr[q]);
                    li[q] = tf32_round(g.y - gi[q]);
                }
                auto row = [&](int n) {
                    return bbuf(b) + (unsigned)quad * KSB + (unsigned)(n >> 3) * 128u + (unsigned)(n & 7) * 16u;
                };
                st_shared_v4(row(k), -gi[0], -gi[1], -gi[2], -gi[3]);
                st_shared_v4(row(NB + k), gr[0], gr[1], gr[2], gr[3]);
                st_shared_v4(row(2 * NB + k), gi[0], gi[1], gi[2], gi[3]);
                if (SPLIT == 3) {
                    st_shared_v4(BPART + row(k), -li[0], -li[1], -li[2], -li[3]);
                    st_shared_v4(BPART + row(NB + k), lr[0], lr[1], lr[2], lr[3]);
                    st_shared_v4(BPART + row(2 * NB + k), li[0], li[1], li[2], li[3]);
                }
            }
        }
    };
    // the MMAs of chunk c from buffer b: per K step of 8 points, [Re D | Im D] +=
    // Kr [Gr | Gi] + Ki [-Gi | Gr] (hi*hi, and hi*lo + lo*hi for SPLIT = 3)
    auto issue = [&](int c, int b, unsigned tmem) {
#pragma unroll
        for (int ks = 0; ks < KC / 8; ++ks) {
            const unsigned bb = bbuf(b) + (unsigned)ks * 2u * KSB;
            const unsigned ar = abuf(b) + (unsigned)ks * 2u * KSA;
            const unsigned long long b1 = smem_desc(bb + (unsigned)(NB / 8) * 128u, KSB, 128u);
            const unsigned long long b2 = smem_desc(bb, KSB, 128u);
            const unsigned long long dre = smem_desc(ar, KSA, 128u);
            const unsigned long long dim = smem_desc(ar + PLANE, KSA, 128u);
            mma_tf32(tmem, dre, b1, IDESC, (c > 0 || ks > 0) ? 1 : 0);
            mma_tf32(tmem, dim, b2, IDESC, 1);
            if (SPLIT == 3) {
                const unsigned long long b1l = smem_desc(BPART + bb + (unsigned)(NB / 8) * 128u, KSB, 128u);
                const unsigned long long b2l = smem_desc(BPART + bb, KSB, 128u);
                mma_tf32(tmem, dre, b1l, IDESC, 1);
                mma_tf32(tmem, dim, b2l, IDESC, 1);
                mma_tf32(tmem, smem_desc(ar + 2u * PLANE, KSA, 128u), b1, IDESC, 1);
                mma_tf32(tmem, smem_desc(ar + 3u * PLANE, KSA, 128u), b2, IDESC, 1);
            }
        }
        mma_commit(&mma_bar[b]);
    };

    T k0[KC], k1[KC], g0[PPT][4], g1[PPT][4], c0[PPT][4], c1[PPT][4];
    tc_fence_before();
    __syncthreads();                                        // row offsets, barriers, tensor memory
    tc_fence_after();
    const unsigned tmem = tmem_base;
    if (nch > 0) load_k(0, k0);                             // K is immutable: before the wait
    asm volatile("griddepcontrol.wait;\n" ::: "memory");    // incoming data, base and sub are ready
    if (nch > 0) load_g(0, g0, c0);
    bool issued = false;
    // one chunk: load chunk c + 1, wait until the MMAs of chunk c - 2 released buffer
    // c % 2, write chunk c, hand it to the MMA thread
    auto step = [&](int c, T (&kc)[KC], T (&gc)[PPT][4], T (&cc)[PPT][4], T (&kn)[KC], T (&gn)[PPT][4],
                    T (&cn)[PPT][4]) -> bool {
        const int b = c & 1;
        if (c + 1 < nch) {
            load_k(c + 1, kn);
            load_g(c + 1, gn, cn);
        }
        if (c >= 2 && !bar_wait(&mma_bar[b], (unsigned)(((c - 2) >> 1) & 1), TC_WAIT_LIMIT)) {
            abort_flag = 1;
            if (a.err) atomicExch(a.err, (int)HELM_ERR_TIMEOUT);
        }
        store(b, kc, gc, cc);
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        tc_fence_before();
        __syncthreads();
        if (abort_flag) return false;
        if (tid == 0) {
            tc_fence_after();
            issue(c, b, tmem);
            issued = true;
        }
        return true;
    };
    bool ok = true;
    for (int c = 0; c < nch && ok; c += 2) {
        ok = step(c, k0, g0, c0, k1, g1, c1);
        if (ok && c + 1 < nch) ok = step(c + 1, k1, g1, c1, k0, g0, c0);
    }
    if (ok && nch > 0) {
        // the last commit arrives when every MMA of the CTA has completed
        if (!bar_wait(&mma_bar[(nch - 1) & 1], (unsigned)(((nch - 1) >> 1) & 1), TC_WAIT_LIMIT)) {
            abort_flag = 1;
            if (a.err) atomicExch(a.err, (int)HELM_ERR_TIMEOUT);
        }
    }
    __syncthreads();
    ok = abort_flag == 0;
    if (!ok && tid == 0 && issued) {
        mma_commit(&fin_bar);
        bar_wait(&fin_bar, 0u, TC_WAIT_LIMIT);
    }
    tc_fence_after();
    __shared__ int last_s;
    if (ok) {
        // row tid's accumulators for the block's RHS (none: this CTA had no chunk)
        float acc[NCOLS];
        const unsigned trow = tmem + ((unsigned)(32 * warp) << 16);
        if (nch > 0) {
#pragma unroll
            for (int cb = 0; cb < NCOLS; cb += 8) tmem_ld8(trow + (unsigned)cb, acc + cb);
            tmem_wait_ld();
        } else {
#pragma unroll
            for (int cc = 0; cc < NCOLS; ++cc) acc[cc] = 0.f;
        }
        bool fin = true;
        if (S > 1) {
            // split tile: every CTA stores its partial sums; the last to arrive adds the S
            // partials in split order (the same sums whichever CTA is last) and finishes
            const long long unit = ((long long)slot * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
            float* pp = a.part + unit * S * (128LL * NCOLS);
#pragma unroll
            for (int cc = 0; cc < NCOLS; ++cc) HST(pp + ((long long)split * NCOLS + cc) * 128 + tid, acc[cc]);
            __threadfence();
            __syncthreads();
            if (tid == 0) {
                const int old = HELM_CHK(a.cnt + unit, sizeof(int)) ? atomicAdd(a.cnt + unit, 1) : -1;
                last_s = old == S - 1;
                if (old == S - 1) HST(a.cnt + unit, 0);     // ready for the next launch
            }
            __syncthreads();
            fin = last_s != 0;
            if (fin) {
                __threadfence();
#pragma unroll
                for (int cc = 0; cc < NCOLS; ++cc) acc[cc] = 0.f;
                for (int sp = 0; sp < S; ++sp)
#pragma unroll
                    for (int cc = 0; cc < NCOLS; ++cc) acc[cc] += HLDCG(pp + ((long long)sp * NCOLS + cc) * 128 + tid);
            }
        }
        if (fin && live) {
            const long long ti = sel(tin, srow) + pt;
            const TraceCoef<T> cf = HLD(a.tc + ti);
            const long long to = (long long)(srow == 0 ? sd.tout[0] : srow == 1 ? sd.tout[1] : srow == 2 ? sd.tout[2]
                                                                                                         : sd.tout[3]) + pt;
#pragma unroll
            for (int k0_ = 0; k0_ < NB; k0_ += 8) {
                T gin[8], bs[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int k = k0_ + u;
                    gin[u] = bs[u] = make_float2(0.f, 0.f);
                    if (k < nr) {
                        const long long oi = (long long)(rhs0 + k) * a.ntrace + ti;
                        const long long o = (long long)(rhs0 + k) * a.ntrace + to;
                        if (a.gin0) gin[u] = HLD(a.gin0 + oi);
                        if (a.gin1) gin[u] = cadd(gin[u], HLD(a.gin1 + oi));
                        if (a.base) bs[u] = HLD(a.base + o);
                        if (a.sub) bs[u] = csub(bs[u], HLD(a.sub + o));
                    }
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int k = k0_ + u;
                    if (k < nr) {
                        const T d = make_float2(acc[k], acc[NB + k]);
                        const T out = cadd(cfma(cf.cb, d, cmul(cf.ca, gin[u])), bs[u]);
                        const long long o = (long long)(rhs0 + k) * a.ntrace + to;
                        HST(a.dst + o, out);
                        if (a.dst2) HST(a.dst2 + o, out);
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TCOLS) : "memory");
    }
}

template <int NB, int SPLIT>
cudaError_t tc_iface_launch(const IfaceArgs<float>& a, int nactive, int max_rows, int S, cudaStream_t st) {
    constexpr size_t smem = 2 * ((SPLIT == 3 ? 4 : 2) * 4 * 2064 + (SPLIT == 3 ? 2 : 1) * 4 * 48 * NB);
    cudaError_t e = cudaFuncSetAttribute(tc_iface_kernel<NB, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((a.nrhs + NB - 1) / NB, (max_rows + 127) / 128, nactive * S);
    cfg.blockDim = dim3(128);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    count_launch();
    return cudaLaunchKernelEx(&cfg, tc_iface_kernel<NB, SPLIT>, a, S);
}

// ------------------------------------------------------------- factorisation
// The block-tridiagonal factorisation of a subdomain (T_1 = D_1, X_r = T_r^{-1},
// T_{r+1} = D_{r+1} - X_r; see k_factor.cu) with the inversions as blocked
// Gauss-Jordan eliminations whose trailing updates run on the tensor cores.
//
// Partial pivoting is virtual: rows stay where they are, the pivot of column k is the
// largest remaining entry of that column, at row p_k.  Columns are taken in panels of
// FB = 16.  A panel is eliminated on the CUDA cores on its own columns only (one row
// per thread of the first four warps): afterwards its pivot rows hold M11^{-1} and the
// other rows -M21 M11^{-1}, where M11 is the panel's block on its pivot rows.  Every
// other column then takes the same row operations, for all rows at once, as the rank-FB
// update
//     W[:, q] += A B[:, q],   A[i, j] = W[i, c + j] - (i == p_{c+j}),   B[j, q] = W_old[p_{c+j}, q]
// (for a pivot row this is M11^{-1} M12, for the others M22 - M21 M11^{-1} M12), with B
// zero on the panel's own columns: a complex (128 x 16) x (16 x 128) product, the
// [-Bi | Br | Bi] operand of the block solves (k_tc.cu above), split into TF32 hi + lo
// (three MMAs per real product), accumulated in tensor memory and added to W by the
// epilogue warps.  At the end X[k][l] = W[p_k][j(l)] with p_{j(l)} = l undoes the
// virtual interchanges; the stored X_r is symmetrised as in k_factor.cu.  One CTA of
// 512 threads per subdomain (at most 128 nodes wide), W in shared memory (row stride
// 129 complex values: conflict-free row and column walks).
constexpr int FB = 16;                                   // panel width (K of the update)
constexpr int FT_TC = 512;                               // threads per CTA
constexpr int LDW = 129;                                 // row stride of W (complex values)
constexpr unsigned F_PLANE = 128u * FB * 4u;             // one plane of the A operand (bytes)
constexpr unsigned F_KSA = 2048u;                        // A: K-adjacent core matrices
constexpr unsigned F_KSB = 48u * 128u + 64u;             // B: K-adjacent core matrices (N = 3 x 128)
constexpr unsigned F_BLO = (FB / 4) * F_KSB;             // offset of the lo B operand
constexpr size_t F_W_BYTES = (size_t)128 * LDW * sizeof(float2);
constexpr size_t F_A_OFF = (F_W_BYTES + 1023) & ~(size_t)1023;
constexpr size_t F_B_OFF = F_A_OFF + 4 * F_PLANE;
constexpr size_t F_SMEM = F_B_OFF + 2 * (size_t)F_BLO;

__global__ void __launch_bounds__(FT_TC, 1) tc_factor_kernel(const SubDev* __restrict__ subtab,
                                                             const double2* __restrict__ dloc, float2* __restrict__ X,
                                                             int* __restrict__ info, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long mma_bar, fin_bar;
    __shared__ unsigned tmem_base;
    __shared__ int piv[128], ipiv[128], used[128];
    __shared__ float2 prow[FB];
    __shared__ float red_v[4];
    __shared__ int red_i[4];
    __shared__ int s_p, abort_flag;
    __shared__ float2 s_inv;
    float2* W = reinterpret_cast<float2*>(smem_raw);
    unsigned char* aop = smem_raw + F_A_OFF;
    unsigned char* bop = smem_raw + F_B_OFF;
    const unsigned a_s = sm_addr(aop), b_s = sm_addr(bop);
    const SubDev sd = subtab[blockIdx.x];
    const int m = sd.mx, my = sd.my;
    const int w0 = sd.w0, ld0 = sd.ld0, ld1 = sd.ld1;
    const long long xr_elems = (long long)m * (ld0 + ld1);
    auto xidx = [&](int i, int j) -> long long {
        return j < w0 ? (long long)i * ld0 + j : (long long)m * ld0 + (long long)i * ld1 + (j - w0);
    };
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr unsigned IDESC = tf32_idesc(256);
    if (tid == 0) {
        bar_init(&mma_bar, 1);
        bar_init(&fin_bar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(sm_addr(&tmem_base)),
                     "r"(256)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = tmem_base;
    int fail_at = 0;                                     // thread 0: first vanishing pivot (1-based)
    unsigned ph = 0;
    bool issued_any = false;

    for (int r = 0; r < my && !abort_flag; ++r) {
        // T_r = D_r - X_{r-1}
        const double2* d = dloc + sd.loff + (long long)r * m;
        const float2* Xp = X + sd.xoff + (long long)(r - 1) * xr_elems;
        for (int idx = tid; idx < m * m; idx += FT_TC) {
            const int i = idx / m, j = idx - i * m;
            float2 v = make_float2(0.f, 0.f);
            if (r > 0) {
                const float2 xp = Xp[xidx(i, j)];
                v = make_float2(-xp.x, -xp.y);
            }
            if (i == j) v = make_float2(v.x + (float)d[i].x, v.y + (float)d[i].y);
            else if (i - j == 1 || j - i == 1) v.x -= 1.f;
            W[i * LDW + j] = v;
        }
        if (tid < 128) used[tid] = 0;
        __syncthreads();
        for (int c = 0; c < m; c += FB) {
            const int nb = min(FB, m - c);
            // ---- the panel's own columns, rows on the first four warps
            if (tid < 128) {
                const int i = tid;
                for (int k = c; k < c + nb; ++k) {
                    float best = -1.f;
                    if (i < m && !used[i]) {
                        const float2 v = W[i * LDW + k];
                        best = v.x * v.x + v.y * v.y;
                    }
                    int bi = i;
                    for (int o = 16; o > 0; o >>= 1) {
                        const float ob = __shfl_down_sync(0xffffffffu, best, o);
                        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
                        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
                    }
                    if (lane == 0) { red_v[warp] = best; red_i[warp] = bi; }
                    asm volatile("bar.sync 1, 128;\n" ::: "memory");
                    if (tid == 0) {
                        float b = red_v[0];
                        int p = red_i[0];
                        for (int q = 1; q < 4; ++q)
                            if (red_v[q] > b || (red_v[q] == b && red_i[q] < p)) { b = red_v[q]; p = red_i[q]; }
                        if (!(b > 0.f) && !fail_at) fail_at = r * m + k + 1;
                        s_p = p;
                        piv[k] = p;
                        used[p] = 1;
                        const float2 pv = W[p * LDW + k];
                        const float dd = pv.x * pv.x + pv.y * pv.y;
                        s_inv = dd > 0.f ? make_float2(pv.x / dd, -pv.y / dd) : make_float2(0.f, 0.f);
                    }
                    asm volatile("bar.sync 1, 128;\n" ::: "memory");
                    const int p = s_p;
                    const float2 inv = s_inv;
                    if (tid < nb) {
                        const int j = c + tid;
                        prow[tid] = j == k ? inv : cmul(W[p * LDW + j], inv);
                    }
                    asm volatile("bar.sync 1, 128;\n" ::: "memory");
                    if (i < m) {
                        if (i == p) {
                            for (int jj = 0; jj < nb; ++jj) W[i * LDW + c + jj] = prow[jj];
                        } else {
                            const float2 f = W[i * LDW + k];
                            for (int jj = 0; jj < nb; ++jj) {
                                const int j = c + jj;
                                W[i * LDW + j] = j == k ? make_float2(-(f.x * inv.x - f.y * inv.y), -(f.x * inv.y + f.y * inv.x))
                                                        : cfma(make_float2(-f.x, -f.y), prow[jj], W[i * LDW + j]);
                            }
                        }
                    }
                    asm volatile("bar.sync 1, 128;\n" ::: "memory");
                }
            }
            __syncthreads();
            // ---- operands of the rank-nb update
            for (int e = tid; e < 128 * FB; e += FT_TC) {
                const int i = e / FB, jj = e - i * FB;
                float2 v = make_float2(0.f, 0.f);
                if (i < m && jj < nb) {
                    v = W[i * LDW + c + jj];
                    if (i == piv[c + jj]) v.x -= 1.f;
                }
                const unsigned off = (unsigned)((((jj >> 2) * 16 + (i >> 3)) * 32 + (i & 7) * 4 + (jj & 3)) * 4);
                const float hr = tf32_round(v.x), hi = tf32_round(v.y);
                *reinterpret_cast<float*>(aop + off) = hr;
                *reinterpret_cast<float*>(aop + F_PLANE + off) = hi;
                *reinterpret_cast<float*>(aop + 2 * F_PLANE + off) = tf32_round(v.x - hr);
                *reinterpret_cast<float*>(aop + 3 * F_PLANE + off) = tf32_round(v.y - hi);
            }
            for (int e = tid; e < FB * 128; e += FT_TC) {
                const int jj = e >> 7, q = e & 127;
                float2 v = make_float2(0.f, 0.f);
                if (jj < nb && q < m && (q < c || q >= c + nb)) v = W[piv[c + jj] * LDW + q];
                const float hr = tf32_round(v.x), hi = tf32_round(v.y);
                const float lr = tf32_round(v.x - hr), li = tf32_round(v.y - hi);
                auto row = [&](int n) {
                    return (unsigned)(jj >> 2) * F_KSB + (unsigned)(n >> 3) * 128u + (unsigned)(n & 7) * 16u +
                           (unsigned)(jj & 3) * 4u;
                };
                *reinterpret_cast<float*>(bop + row(q)) = -hi;
                *reinterpret_cast<float*>(bop + row(128 + q)) = hr;
                *reinterpret_cast<float*>(bop + row(256 + q)) = hi;
                *reinterpret_cast<float*>(bop + F_BLO + row(q)) = -li;
                *reinterpret_cast<float*>(bop + F_BLO + row(128 + q)) = lr;
                *reinterpret_cast<float*>(bop + F_BLO + row(256 + q)) = li;
            }
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            tc_fence_before();
            __syncthreads();
            // ---- [Re D | Im D] = Ar [Br | Bi] + Ai [-Bi | Br], 3xTF32
            if (tid == 0) {
                tc_fence_after();
#pragma unroll
                for (int kk = 0; kk < FB / 8; ++kk) {
                    const unsigned ar = a_s + (unsigned)kk * 2u * F_KSA;
                    const unsigned bb = b_s + (unsigned)kk * 2u * F_KSB;
                    const unsigned long long dre = smem_desc(ar, F_KSA, 128u);
                    const unsigned long long dim = smem_desc(ar + F_PLANE, F_KSA, 128u);
                    const unsigned long long drel = smem_desc(ar + 2u * F_PLANE, F_KSA, 128u);
                    const unsigned long long diml = smem_desc(ar + 3u * F_PLANE, F_KSA, 128u);
                    const unsigned long long b1 = smem_desc(bb + 16u * 128u, F_KSB, 128u);
                    const unsigned long long b2 = smem_desc(bb, F_KSB, 128u);
                    const unsigned long long b1l = smem_desc(F_BLO + bb + 16u * 128u, F_KSB, 128u);
                    const unsigned long long b2l = smem_desc(F_BLO + bb, F_KSB, 128u);
                    mma_tf32(tmem, dre, b1, IDESC, kk > 0 ? 1 : 0);
                    mma_tf32(tmem, dim, b2, IDESC, 1);
                    mma_tf32(tmem, dre, b1l, IDESC, 1);
                    mma_tf32(tmem, dim, b2l, IDESC, 1);
                    mma_tf32(tmem, drel, b1, IDESC, 1);
                    mma_tf32(tmem, diml, b2, IDESC, 1);
                }
                mma_commit(&mma_bar);
                issued_any = true;
            }
            if (!bar_wait(&mma_bar, ph, TC_WAIT_LIMIT)) {
                if (threadIdx.x == 0) {
                    abort_flag = 1;
                    if (err) atomicExch(err, (int)HELM_ERR_TIMEOUT);
                }
            }
            ph ^= 1u;
            tc_fence_after();
            // ---- W += D: warp w reads TMEM lanes 32 (w & 3) .. (rows) and columns 32 (w >> 2) ..
            {
                const int qr = warp & 3, g = warp >> 2;
                const int i = 32 * qr + lane;
                const unsigned base = tmem + ((unsigned)(32 * qr) << 16) + (unsigned)(32 * g);
                float dr[32], di[32];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    tmem_ld8(base + (unsigned)(8 * t), dr + 8 * t);
                    tmem_ld8(base + 128u + (unsigned)(8 * t), di + 8 * t);
                }
                tmem_wait_ld();
                if (i < m && !abort_flag) {
#pragma unroll
                    for (int t = 0; t < 32; ++t) {
                        const int q = 32 * g + t;
                        if (q < m) {
                            float2 w = W[i * LDW + q];
                            w.x += dr[t];
                            w.y += di[t];
                            W[i * LDW + q] = w;
                        }
                    }
                }
            }
            tc_fence_before();
            __syncthreads();
            if (abort_flag) break;
        }
        if (abort_flag) break;
        // X_r: undo the virtual interchanges, symmetrise, two-half layout with zeroed padding
        if (tid < m) ipiv[piv[tid]] = tid;
        __syncthreads();
        float2* Xr = X + sd.xoff + (long long)r * xr_elems;
        for (long long idx = tid; idx < xr_elems; idx += FT_TC) {
            int i, j;
            bool pad;
            if (idx < (long long)m * ld0) {
                i = (int)(idx / ld0);
                j = (int)(idx - (long long)i * ld0);
                pad = j >= w0;
            } else {
                const long long t2 = idx - (long long)m * ld0;
                i = (int)(t2 / ld1);
                j = w0 + (int)(t2 - (long long)i * ld1);
                pad = j >= m;
            }
            float2 v = make_float2(0.f, 0.f);
            if (!pad) {
                const float2 a = W[piv[i] * LDW + ipiv[j]], b = W[piv[j] * LDW + ipiv[i]];
                v = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y + b.y));
            }
            Xr[idx] = v;
        }
        __syncthreads();
    }
    // no MMA of this CTA is in flight when tensor memory is freed (bounded)
    if (tid == 0 && issued_any) {
        mma_commit(&fin_bar);
        bar_wait(&fin_bar, 0u, TC_WAIT_LIMIT);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(256) : "memory");
    }
    if (tid == 0) info[blockIdx.x] = fail_at;
}

}  // namespace

int tc_tiles(int mx) { return mx <= 128 ? 1 : mx <= 256 ? 2 : 0; }

long long tc_layout_floats(int mx, int my, int MT, int split) {
    const int KC = tc_kc(MT, split);
    return (long long)my * ((mx + KC - 1) / KC) * (TC_CHUNK_BYTES / 4);
}

cudaError_t launch_tc_layout(const SubDev* subtab, int nsub, int split, const float2* X, float* XT, cudaStream_t st) {
    if (nsub == 0) return cudaSuccess;
    count_launch();
    tc_layout_kernel<<<dim3(64, nsub), 256, 0, st>>>(subtab, nsub, split, X, XT);
    return cudaGetLastError();
}

// RHS per CTA: the widest block whose operands fit next to a ring of chunk slots
cudaError_t launch_tc_stage(const StageArgs<float>& a, const float* XT, int MT, int split, int nactive,
                            cudaStream_t st, int nr) {
    if (nactive == 0) return cudaSuccess;
    const int n = a.nrhs;
    // RHS per CTA: the largest variant that the RHS count fills (or the tuned one)
    auto want = [&](int v) { return nr > 0 ? nr == v : n >= v; };
    if (split == 3) {
        if (MT == 1) {
            if (want(32) && n >= 32) return tc_launch<1, 32, false, 3>(a, XT, nactive, (n + 31) / 32, st);
            return tc_launch<1, 16, false, 3>(a, XT, nactive, (n + 15) / 16, st);
        }
        if (MT == 2) return tc_launch<2, 16, false, 3>(a, XT, nactive, (n + 15) / 16, st);
        return cudaErrorInvalidValue;
    }
    if (MT == 1) {
        if (want(64) && n >= 64) return tc_launch<1, 64, false, 1>(a, XT, nactive, (n + 63) / 64, st);
        if (want(32) && n >= 32) return tc_launch<1, 32, false, 1>(a, XT, nactive, (n + 31) / 32, st);
        return tc_launch<1, 16, false, 1>(a, XT, nactive, (n + 15) / 16, st);
    }
    if (MT == 2) {
        if (want(32) && n >= 32) return tc_launch<2, 32, false, 1>(a, XT, nactive, (n + 31) / 32, st);
        return tc_launch<2, 16, false, 1>(a, XT, nactive, (n + 15) / 16, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_tc_basis(const StageArgs<float>& a, const float* XT, int MT, int split, int nsub, int ncols,
                            cudaStream_t st) {
    if (nsub == 0) return cudaSuccess;
    if (split == 3) {
        if (MT == 1) return tc_launch<1, 32, true, 3>(a, XT, nsub, (ncols + 31) / 32, st);
        if (MT == 2) return tc_launch<2, 16, true, 3>(a, XT, nsub, (ncols + 15) / 16, st);
        return cudaErrorInvalidValue;
    }
    if (MT == 1) return tc_launch<1, 64, true, 1>(a, XT, nsub, (ncols + 63) / 64, st);
    if (MT == 2) return tc_launch<2, 32, true, 1>(a, XT, nsub, (ncols + 31) / 32, st);
    return cudaErrorInvalidValue;
}

// an interface stage with 16 or more RHS on the tensor cores (see tc_iface_kernel); a
// stage of fewer than min_ctas output tiles splits each tile's boundary points over up
// to 8 CTAs (when the partial-sum scratch holds them) so that it makes about that many
cudaError_t launch_iface_tc(const IfaceArgs<float>& a, int nactive, int max_rows, int split, int nb, int min_ctas,
                            int max_Lb, cudaStream_t st) {
    if (nactive == 0 || a.nrhs == 0 || max_rows == 0) return cudaSuccess;
    const long long tiles = (long long)nactive * ((max_rows + 127) / 128) * ((a.nrhs + nb - 1) / nb);
    int S = 1;
    if (a.part && a.cnt && tiles < min_ctas) {
        S = (int)std::min<long long>(8, (min_ctas + tiles - 1) / tiles);
        S = std::min(S, std::max(1, (max_Lb + 15) / 16));
        while (S > 1 && (tiles > a.cnt_cap || tiles * S * 128LL * 2 * (nb >= 32 ? 32 : 16) > a.part_cap)) --S;
    }
    if ((long long)nactive * S > 65535) return cudaErrorInvalidValue;
    if (split == 3) return nb >= 32 ? tc_iface_launch<32, 3>(a, nactive, max_rows, S, st)
                                    : tc_iface_launch<16, 3>(a, nactive, max_rows, S, st);
    return nb >= 32 ? tc_iface_launch<32, 1>(a, nactive, max_rows, S, st)
                    : tc_iface_launch<16, 1>(a, nactive, max_rows, S, st);
}

// The complex64 factorisation with the tensor-core trailing updates (tc_factor_kernel);
// every subdomain at most 128 nodes wide.
cudaError_t launch_tc_factor(const SubDev* subtab, int nsub, const double2* dloc, float2* X, int* info, int* err,
                             cudaStream_t st) {
    if (nsub == 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(tc_factor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)F_SMEM);
    if (e != cudaSuccess) return e;
    count_launch();
    tc_factor_kernel<<<nsub, FT_TC, F_SMEM, st>>>(subtab, dloc, X, info, err);
    return cudaGetLastError();
}
