// The Pade HABC transmission (Sections 3 and 6: high-order absorbing conditions as
// the transmission conditions, N_pade auxiliary fields, rotation phi) on the GPU.
//
// On an interface side of L points the condition (d_n - T) u = g has the dense
// operator T = i diag(k) e^{i phi/2} R_N(W), W = (I + diag(1/k^2) Lap) e^{-i phi} - I,
// R_N(W) = I + sum_l a_l (I + b_l W)^{-1} W (the rotated-branch [N/N] Pade square
// root; Lap the 3-point second difference along the side with Neumann ends, k the
// edge wavenumber of each point).  With B = T h/2 the mid-edge ghost relation gives
//     local right-hand side  Rin G,            Rin = (I - B)^{-1},
//     local matrix block     -(2 Rin - I)      (in place of the scalar Robin c0),
//     outgoing data          M1 u_p + M2 G,    M1 = 4 (I - Rin),  M2 = I - 2 Rin.
//
// The library keeps the block-tridiagonal factors of a base problem with the
// scalar optimized Robin condition (c0 per point) and folds the HABC side blocks
// in through the interface boundary space (Woodbury): with K the boundary block of
// the base inverse and C = blockdiag(2 Rin_s - I) - diag(c0),
//     K_HABC = W K,  W = (I - K C)^{-1},
// and per subdomain, with P1 = W K Rin (all on the Lb boundary points):
//     interface stage   G_out = Q G,               Q  = M1 P1 + M2
//     lifting           G_out = Lq u_f,            Lq = M1 W       (u_f: base solve of the source)
//     reconstruction    base solve with datum      D1 G + D2 u_f,  D1 = Rin + C P1,  D2 = C W.
// Since M1, M2 and C are affine in Rin, only Rin P1 and Rin W are needed besides W
// and P1.  Everything here runs once per factorisation (setup of the transmission)
// in FP64: the side operators (tridiagonal solves with partial pivoting, one
// column per thread), a cooperative Gauss-Jordan inversion with partial pivoting
// (columns spread over all SMs in shared memory, one grid barrier per pivot), a
// batched complex GEMM and elementwise combinations.
#include "helm_internal.cuh"

#include <algorithm>

namespace {

constexpr int HT = 256;                              // threads per CTA
constexpr double kPi = 3.14159265358979323846;
constexpr long long GJ_WAIT = 2000000000LL;          // cycles (~1 s) before a grid barrier gives up

__device__ __forceinline__ double2 cdivd(double2 a, double2 b) {
    const double s = fabs(b.x) + fabs(b.y);
    const double br = b.x / s, bi = b.y / s, ar = a.x / s, ai = a.y / s;
    const double d = br * br + bi * bi;
    return make_double2((ar * br + ai * bi) / d, (ai * br - ar * bi) / d);
}
__device__ __forceinline__ double cabs1(double2 a) { return fabs(a.x) + fabs(a.y); }

// ------------------------------------------------------------ side operators
// One CTA per interface slot (subdomain i, side toward j): kappa_e of its points, then
// for every Pade term the tridiagonal I + b_l W factored with adjacent-row pivoting
// (thread 0) and solved for every unit column (one column per thread, the column kept
// in Y, rows coalesced across threads), R accumulated in M, and finally
// M = I - (h/2) T.  Y and M are L x L row-major at the slot's matrix offset.
__global__ void __launch_bounds__(HT) habc_side_kernel(const double* __restrict__ m2, int nx, double h, double omega,
                                                      int n_pade, double phi, const int* __restrict__ slot_sub,
                                                      const int* __restrict__ slot_side,
                                                      const int* __restrict__ slot_len,
                                                      const long long* __restrict__ slot_moff,
                                                      const SubDev* __restrict__ subtab, double2* __restrict__ M,
                                                      double2* __restrict__ Y) {
    extern __shared__ double2 sh[];
    const int slot = blockIdx.x;
    const SubDev sd = subtab[slot_sub[slot]];
    const int side = slot_side[slot], L = slot_len[slot];
    double2* d = sh;            // [L] diagonal of U
    double2* du = d + L;        // [L] first superdiagonal of U
    double2* du2 = du + L;      // [L] second superdiagonal of U (from interchanges)
    double2* ml = du2 + L;      // [L] multipliers
    double* kap = reinterpret_cast<double*>(ml + L);     // [L] kappa_e
    int* swp = reinterpret_cast<int*>(kap + L);          // [L] 1: rows i and i+1 were interchanged
    double2* Ms = M + slot_moff[slot];
    double2* Ys = Y + slot_moff[slot];
    for (int k = threadIdx.x; k < L; k += HT) {
        int ap, bp, aq, bq;
        if (side == SW || side == SE) {
            bp = bq = sd.y0 + k;
            ap = side == SW ? sd.x0 : sd.x0 + sd.mx - 1;
            aq = side == SW ? ap - 1 : ap + 1;
        } else {
            ap = aq = sd.x0 + k;
            bp = side == SS ? sd.y0 : sd.y0 + sd.my - 1;
            bq = side == SS ? bp - 1 : bp + 1;
        }
        kap[k] = omega * sqrt(0.5 * (m2[(long long)bp * nx + ap] + m2[(long long)bq * nx + aq]));
    }
    for (long long e = threadIdx.x; e < (long long)L * L; e += HT)
        Ms[e] = make_double2((e / L == e % L) ? 1.0 : 0.0, 0.0);      // R starts as I
    __syncthreads();
    const double2 rot = make_double2(cos(phi), -sin(phi));           // e^{-i phi}
    const int M2 = 2 * n_pade + 1;
    for (int l = 1; l <= n_pade; ++l) {
        const double th = l * kPi / M2;
        const double al = 2.0 / M2 * sin(th) * sin(th), bl = cos(th) * cos(th);
        if (threadIdx.x == 0) {
            // I + b_l W: W_ii = (1 + s_i (-2 + ends_i)) e^{-i phi} - 1, W_i,i+-1 = s_i e^{-i phi}
            for (int i = 0; i < L; ++i) {
                const double s = 1.0 / (kap[i] * kap[i] * h * h);
                const int ends = (i == 0) + (i == L - 1);
                const double w = 1.0 + s * (-2.0 + ends);
                d[i] = make_double2(1.0 + bl * (w * rot.x - 1.0), bl * w * rot.y);
                du[i] = make_double2(bl * s * rot.x, bl * s * rot.y);       // row i, column i + 1
                ml[i] = make_double2(bl * s * rot.x, bl * s * rot.y);       // row i + 1, column i (row i+1's s below)
                du2[i] = make_double2(0.0, 0.0);
                swp[i] = 0;
            }
            for (int i = 0; i + 1 < L; ++i) {
                const double s1 = 1.0 / (kap[i + 1] * kap[i + 1] * h * h);
                ml[i] = make_double2(bl * s1 * rot.x, bl * s1 * rot.y);     // the subdiagonal entry of row i + 1
            }
            // Gaussian elimination of the subdiagonal, interchanging rows i and i + 1 when
            // the subdiagonal entry is the larger pivot candidate
            for (int i = 0; i + 1 < L; ++i) {
                const double2 sub = ml[i];
                if (cabs1(d[i]) >= cabs1(sub)) {
                    const double2 f = cabs1(d[i]) > 0.0 ? cdivd(sub, d[i]) : make_double2(0.0, 0.0);
                    ml[i] = f;
                    d[i + 1] = csub(d[i + 1], cmul(f, du[i]));
                } else {
                    const double2 f = cdivd(d[i], sub);
                    const double2 di1 = d[i + 1];
                    d[i] = sub;
                    ml[i] = f;
                    const double2 t = du[i];
                    du[i] = di1;
                    d[i + 1] = csub(t, cmul(f, di1));
                    if (i + 2 < L) {
                        du2[i] = du[i + 1];
                        du[i + 1] = make_double2(-(f.x * du[i + 1].x - f.y * du[i + 1].y),
                                                 -(f.x * du[i + 1].y + f.y * du[i + 1].x));
                    }
                    swp[i] = 1;
                }
            }
        }
        __syncthreads();
        // column c of (I + b_l W)^{-1}: forward elimination of e_c, back substitution
        for (int c = threadIdx.x; c < L; c += HT) {
            for (int i = 0; i < L; ++i) Ys[(long long)i * L + c] = make_double2(i == c ? 1.0 : 0.0, 0.0);
            for (int i = 0; i + 1 < L; ++i) {
                const double2 bi = Ys[(long long)i * L + c], bi1 = Ys[(long long)(i + 1) * L + c];
                if (!swp[i]) {
                    Ys[(long long)(i + 1) * L + c] = csub(bi1, cmul(ml[i], bi));
                } else {
                    Ys[(long long)i * L + c] = bi1;
                    Ys[(long long)(i + 1) * L + c] = csub(bi, cmul(ml[i], bi1));
                }
            }
            for (int i = L - 1; i >= 0; --i) {
                double2 v = Ys[(long long)i * L + c];
                if (i + 1 < L) v = csub(v, cmul(du[i], Ys[(long long)(i + 1) * L + c]));
                if (i + 2 < L) v = csub(v, cmul(du2[i], Ys[(long long)(i + 2) * L + c]));
                Ys[(long long)i * L + c] = cdivd(v, d[i]);
            }
            // R += a_l W (I + b_l W)^{-1} = (a_l / b_l) (I - (I + b_l W)^{-1})
            const double q = al / bl;
            for (int i = 0; i < L; ++i) {
                const double2 y = Ys[(long long)i * L + c];
                double2& r = Ms[(long long)i * L + c];
                r.x += q * ((i == c ? 1.0 : 0.0) - y.x);
                r.y += q * (-y.y);
            }
        }
        __syncthreads();
    }
    // M = I - (h/2) T,  T = i e^{i phi/2} diag(k) R
    const double2 pre = make_double2(-sin(0.5 * phi), cos(0.5 * phi));   // i e^{i phi/2}
    for (long long e = threadIdx.x; e < (long long)L * L; e += HT) {
        const int i = (int)(e / L), c = (int)(e % L);
        const double2 t = cmul(pre, cscale(Ms[e], kap[i]));
        Ms[e] = make_double2((i == c ? 1.0 : 0.0) - 0.5 * h * t.x, -0.5 * h * t.y);
    }
}

// ------------------------------------------------------------ Gauss-Jordan
// In-place inversion of a batch of n x n complex matrices (row-major, leading
// dimension lda) by Gauss-Jordan elimination with partial pivoting, one matrix after
// the other, every matrix spread over the whole cooperative grid: CTA b keeps columns
// [b cpb, (b+1) cpb) in shared memory (column-major).  Pivot step k: the owner of
// column k has published that column (after step k-1) and its pivot row; every CTA
// interchanges rows k and p in its columns and eliminates; then the owner of column
// k+1 publishes it.  One grid barrier per step; the published column alternates
// between two buffers.  The row interchanges are undone at the end as column
// interchanges in reverse order.  info[m] = k + 1 when pivot k of matrix m vanished.
struct GjMat {
    double2* A;
    int n, lda;
};

__device__ bool gj_barrier(unsigned* bar, int* err, int* sflag) {
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned g, arrived;
        asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(g) : "l"(bar + 1) : "memory");
        asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(arrived) : "l"(bar) : "memory");
        if (arrived == gridDim.x - 1) {
            asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(bar), "r"(0u) : "memory");
            asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(bar + 1), "r"(g + 1) : "memory");
        } else {
            const long long t0 = clock64();
            unsigned cur;
            do {
                asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(cur) : "l"(bar + 1) : "memory");
                if (cur == g && clock64() - t0 > GJ_WAIT) {
                    atomicExch(err, (int)HELM_ERR_TIMEOUT);
                    *sflag = 1;
                    break;
                }
            } while (cur == g);
        }
    }
    __syncthreads();
    return *sflag == 0;
}

// pub: 2 x (maxn + 2) values: column values, then the pivot row index (as .x)
__global__ void __launch_bounds__(HT, 1) gj_inverse_kernel(const GjMat* __restrict__ mats, int nmat,
                                                           double2* pub, unsigned* bar, int* err, int* info,
                                                           int maxn) {
    extern __shared__ double2 S[];                    // [cpb][n] owned columns, column-major
    __shared__ int sflag;
    __shared__ double rv[HT / 32];
    __shared__ int ri[HT / 32];
    __shared__ int piv_s[1024 + 8];                     // pivot row of every step (n <= 1024)
    __shared__ int idx_s[1024 + 8];
    if (threadIdx.x == 0) sflag = 0;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int P = maxn + 2;
    for (int m = 0; m < nmat; ++m) {
        const GjMat mt = mats[m];
        const int n = mt.n;
        const int cpb = (n + gridDim.x - 1) / gridDim.x;
        const int c0 = blockIdx.x * cpb, c1 = min(n, c0 + cpb);
        for (int jl = 0; jl < c1 - c0; ++jl)
            for (int i = threadIdx.x; i < n; i += HT) S[(long long)jl * n + i] = mt.A[(long long)i * mt.lda + c0 + jl];
        __syncthreads();
        // publish column j (owned here) and its pivot row among rows >= j
        auto publish = [&](int j) {
            const double2* col = S + (long long)(j - c0) * n;
            double2* out = pub + (long long)(j & 1) * P;
            double best = -1.0;
            int bi = j;
            for (int i = threadIdx.x; i < n; i += HT) {
                const double2 v = col[i];
                out[i] = v;
                if (i >= j) {
                    const double a = cabs1(v);
                    if (a > best) { best = a; bi = i; }
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const double ob = __shfl_down_sync(0xffffffffu, best, o);
                const int oi = __shfl_down_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (lane == 0) { rv[warp] = best; ri[warp] = bi; }
            __syncthreads();
            if (threadIdx.x == 0) {
                double b = rv[0];
                int k = ri[0];
                for (int q = 1; q < HT / 32; ++q)
                    if (rv[q] > b || (rv[q] == b && ri[q] < k)) { b = rv[q]; k = ri[q]; }
                out[n] = make_double2((double)k, b);
            }
        };
        if (c0 <= 0 && 0 < c1) publish(0);
        if (!gj_barrier(bar, err, &sflag)) return;
        for (int k = 0; k < n; ++k) {
            const double2* col = pub + (long long)(k & 1) * P;
            const int p = (int)__ldcg(&col[n].x);
            if (threadIdx.x == 0) piv_s[k] = p;
            const double2 ck = __ldcg(&col[k]), cp = __ldcg(&col[p]);
            const double2 pv = cp;                                        // the pivot (row p moves to k)
            const bool sing = cabs1(pv) == 0.0;
            if (sing && blockIdx.x == 0 && threadIdx.x == 0 && info[m] == 0) info[m] = k + 1;
            const double2 inv = sing ? make_double2(0.0, 0.0) : cdivd(make_double2(1.0, 0.0), pv);
            for (int jl = 0; jl < c1 - c0; ++jl) {
                double2* a = S + (long long)jl * n;
                const int j = c0 + jl;
                __syncthreads();
                if (j == k) {
                    // the pivot column becomes column k of the inverse (of the interchanged matrix)
                    for (int i = threadIdx.x; i < n; i += HT) {
                        const double2 ci = i == k ? cp : (i == p ? ck : __ldcg(&col[i]));
                        a[i] = i == k ? inv : make_double2(-(ci.x * inv.x - ci.y * inv.y), -(ci.x * inv.y + ci.y * inv.x));
                    }
                } else {
                    const double2 ak = a[k], ap = a[p];
                    const double2 t = cmul(p == k ? ak : ap, inv);           // new row k entry
                    __syncthreads();
                    for (int i = threadIdx.x; i < n; i += HT) {
                        if (i == k) { a[i] = t; continue; }
                        const double2 ci = i == p ? ck : __ldcg(&col[i]);
                        const double2 ai = (i == p) ? ak : a[i];
                        a[i] = make_double2(ai.x - (ci.x * t.x - ci.y * t.y), ai.y - (ci.x * t.y + ci.y * t.x));
                    }
                }
            }
            __syncthreads();
            if (k + 1 < n && c0 <= k + 1 && k + 1 < c1) publish(k + 1);
            if (!gj_barrier(bar, err, &sflag)) return;
        }
        // undo the interchanges: for l = n-1 .. 0, columns l and piv[l] trade places
        if (threadIdx.x == 0) {
            for (int q = 0; q < n; ++q) idx_s[q] = q;
            for (int l = n - 1; l >= 0; --l) {
                const int t = idx_s[l];
                idx_s[l] = idx_s[piv_s[l]];
                idx_s[piv_s[l]] = t;
            }
        }
        __syncthreads();
        for (int q = 0; q < n; ++q) {
            const int src = idx_s[q];
            if (src < c0 || src >= c1) continue;
            const double2* a = S + (long long)(src - c0) * n;
            for (int i = threadIdx.x; i < n; i += HT) mt.A[(long long)i * mt.lda + q] = a[i];
        }
        // every CTA has written its columns before the next matrix is loaded
        if (!gj_barrier(bar, err, &sflag)) return;
    }
}

// ------------------------------------------------------------ batched GEMM
// C = alpha A B (+ C when accumulate) for a table of complex FP64 problems (row-major,
// leading dimensions per problem).  64 x 64 output tiles, K in chunks of 16, each of
// the 256 threads 4 x 4 outputs.
struct GemmProb {
    const double2* A;
    const double2* B;
    double2* C;
    int m, n, k, lda, ldb, ldc;
    double2 alpha;
    int accumulate;
};

constexpr int GB = 64, GK = 16;

__global__ void __launch_bounds__(256) zgemm_batched_kernel(const GemmProb* __restrict__ probs) {
    const GemmProb pr = probs[blockIdx.y];
    const int tiles_n = (pr.n + GB - 1) / GB;
    const int tm = blockIdx.x / tiles_n, tn = blockIdx.x % tiles_n;
    if (tm * GB >= pr.m) return;
    __shared__ double2 As[GK][GB + 1];
    __shared__ double2 Bs[GK][GB + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = make_double2(0.0, 0.0);
    const int row0 = tm * GB, col0 = tn * GB;
    for (int k0 = 0; k0 < pr.k; k0 += GK) {
        for (int e = threadIdx.x; e < GB * GK; e += 256) {
            const int r = e / GK, kk = e % GK;                 // A tile: row r, column kk
            const int gr = row0 + r, gk = k0 + kk;
            As[kk][r] = (gr < pr.m && gk < pr.k) ? pr.A[(long long)gr * pr.lda + gk] : make_double2(0.0, 0.0);
            const int kb = e / GB, c = e % GB;                 // B tile: row kb, column c
            const int gkb = k0 + kb, gc = col0 + c;
            Bs[kb][c] = (gkb < pr.k && gc < pr.n) ? pr.B[(long long)gkb * pr.ldb + gc] : make_double2(0.0, 0.0);
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < GK; ++kk) {
            double2 a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = cfma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int r = row0 + ty + 16 * i, c = col0 + tx + 16 * j;
            if (r < pr.m && c < pr.n) {
                double2 v = cmul(pr.alpha, acc[i][j]);
                double2* dst = pr.C + (long long)r * pr.ldc + c;
                if (pr.accumulate) v = cadd(v, *dst);
                *dst = v;
            }
        }
}

// ------------------------------------------------------------ assembly
// per subdomain of the batch: its boundary point e lies on side s(e) at point pt(e)
struct HabcSub {
    long long koff;            // element offset of its Lb x Lb operators in the factor-layout arrays
    long long toff;            // element offset of its Lb x Lb temporaries
    int Lb;
    int bo[4], len[4];         // boundary offsets and lengths per side (-1 / 0: outer side)
    long long moff[4];         // offsets of the side matrices Rin_s (slot tin[s]) in the slot-matrix array
    int tin[4];                // trace offsets of the sides (for c0)
};

__device__ __forceinline__ int side_of(const HabcSub& s, int e, int& pt) {
    int sd = 0;
#pragma unroll
    for (int q = 1; q < 4; ++q)
        if (s.bo[q] >= 0 && e >= s.bo[q]) sd = q;
    if (s.bo[0] < 0 && sd == 0) {
        for (int q = 1; q < 4; ++q)
            if (s.bo[q] >= 0) { sd = q; break; }
    }
    pt = e - s.bo[sd];
    return sd;
}

// K (factor precision) -> K64; M = I - 2 K Rin + K + K diag(c0)  (i.e. I - K C) into W
template <typename T>
__global__ void habc_form_kernel(const HabcSub* __restrict__ subs, const T* __restrict__ K,
                                 const TraceCoef<double2>* __restrict__ tc, double2* __restrict__ K64,
                                 const double2* __restrict__ KR, double2* __restrict__ W, int phase) {
    const HabcSub s = subs[blockIdx.y];
    const long long LL = (long long)s.Lb * s.Lb;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < LL; e += (long long)gridDim.x * blockDim.x) {
        if (phase == 0) {
            const T v = HLD(K + s.koff + e);
            HST(K64 + s.toff + e, make_double2((double)v.x, (double)v.y));
        } else {
            const int r = (int)(e / s.Lb), c = (int)(e % s.Lb);
            int pt;
            const int sd = side_of(s, c, pt);
            const double2 ca = HLD(tc + s.tin[sd] + pt).ca;      // c0 = -ca of the base Robin condition
            const double2 k = HLD(K64 + s.toff + e), kr = HLD(KR + s.toff + e);
            // I - K C with C = 2 Rin - I - diag(c0):  I - 2 K Rin + K + K diag(c0)
            const double2 kc0 = cmul(k, make_double2(-ca.x, -ca.y));
            HST(W + s.toff + e, make_double2((r == c ? 1.0 : 0.0) - 2.0 * kr.x + k.x + kc0.x, -2.0 * kr.y + k.y + kc0.y));
        }
    }
}

// Q, Lq, D1, D2 from P1 = W K Rin, RP = Rin P1, W, RW = Rin W (block-diagonal Rin)
template <typename T>
__global__ void habc_final_kernel(const HabcSub* __restrict__ subs, const double2* __restrict__ Mside,
                                  const TraceCoef<double2>* __restrict__ tc, const double2* __restrict__ P1,
                                  const double2* __restrict__ RP, const double2* __restrict__ W,
                                  const double2* __restrict__ RW, T* __restrict__ Q, T* __restrict__ Lq,
                                  T* __restrict__ D1, T* __restrict__ D2) {
    const HabcSub s = subs[blockIdx.y];
    const long long LL = (long long)s.Lb * s.Lb;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < LL; e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / s.Lb), c = (int)(e % s.Lb);
        int pr, pc;
        const int sr = side_of(s, r, pr), sc = side_of(s, c, pc);
        const double2 rin = sr == sc ? HLD(Mside + s.moff[sr] + (long long)pr * s.len[sr] + pc) : make_double2(0.0, 0.0);
        const double2 ca = HLD(tc + s.tin[sr] + pr).ca;
        const double2 c0 = make_double2(-ca.x, -ca.y);
        const double2 p1 = HLD(P1 + s.toff + e), rp = HLD(RP + s.toff + e), w = HLD(W + s.toff + e),
                      rw = HLD(RW + s.toff + e);
        const double id = r == c ? 1.0 : 0.0;
        const double2 q = make_double2(4.0 * (p1.x - rp.x) + id - 2.0 * rin.x, 4.0 * (p1.y - rp.y) - 2.0 * rin.y);
        const double2 lq = make_double2(4.0 * (w.x - rw.x), 4.0 * (w.y - rw.y));
        const double2 c0p = cmul(c0, p1), c0w = cmul(c0, w);
        const double2 d1 = make_double2(rin.x + 2.0 * rp.x - p1.x - c0p.x, rin.y + 2.0 * rp.y - p1.y - c0p.y);
        const double2 d2 = make_double2(2.0 * rw.x - w.x - c0w.x, 2.0 * rw.y - w.y - c0w.y);
        HST(Q + s.koff + e, from_c128<T>(q));
        HST(Lq + s.koff + e, from_c128<T>(lq));
        HST(D1 + s.koff + e, from_c128<T>(d1));
        HST(D2 + s.koff + e, from_c128<T>(d2));
    }
}

// out[k ntrace + t] = in[k ntrace + swp[t]]: slot (i, j) <-> slot (j, i), point by point
template <typename T>
__global__ void trace_swap_kernel(const T* __restrict__ in, T* __restrict__ out, const int* __restrict__ swp,
                                  long long ntrace, int nrhs) {
    const long long tot = ntrace * nrhs;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const long long k = e / ntrace, t = e - k * ntrace;
        HST(out + e, HLD(in + k * ntrace + HLD(swp + t)));
    }
}

}  // namespace

// ------------------------------------------------------------------ launchers
cudaError_t launch_habc_sides(const double* m2, int nx, double h, double omega, int n_pade, double phi,
                              const int* slot_sub, const int* slot_side, const int* slot_len,
                              const long long* slot_moff, int nslots, int max_len, const SubDev* subtab, double2* M,
                              double2* Y, cudaStream_t st) {
    if (nslots == 0) return cudaSuccess;
    const size_t smem = (size_t)max_len * (4 * sizeof(double2) + sizeof(double) + sizeof(int));
    cudaError_t e = cudaFuncSetAttribute(habc_side_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    count_launch();
    habc_side_kernel<<<nslots, HT, smem, st>>>(m2, nx, h, omega, n_pade, phi, slot_sub, slot_side, slot_len, slot_moff,
                                               subtab, M, Y);
    return cudaGetLastError();
}

// CTAs of the cooperative inversion and the largest order it takes
int gj_grid(int maxn) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))
        return 0;
    const int cpb = (maxn + sms - 1) / sms;
    if (maxn > 1024 || (size_t)cpb * maxn * sizeof(double2) > 200 * 1024) return 0;
    return sms;
}

// host: mats (device array of nmat GjMat), pub 2 (maxn + 2) values, bar two zeroed words, info nmat ints (zeroed)
cudaError_t launch_gj_inverse(const void* mats, int nmat, int maxn, double2* pub, unsigned* bar, int* err, int* info,
                              cudaStream_t st) {
    const int grid = gj_grid(maxn);
    if (grid <= 0) return cudaErrorInvalidValue;
    const int cpb = (maxn + grid - 1) / grid;
    const size_t smem = (size_t)cpb * maxn * sizeof(double2);
    cudaError_t e = cudaFuncSetAttribute(gj_inverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const GjMat* m = (const GjMat*)mats;
    void* args[] = {(void*)&m, (void*)&nmat, (void*)&pub, (void*)&bar, (void*)&err, (void*)&info, (void*)&maxn};
    count_launch();
    return cudaLaunchCooperativeKernel((const void*)gj_inverse_kernel, dim3(grid), dim3(HT), args, smem, st);
}
size_t gj_mat_bytes() { return sizeof(GjMat); }
void gj_mat_fill(void* dst, int i, double2* A, int n, int lda) { ((GjMat*)dst)[i] = GjMat{A, n, lda}; }

size_t gemm_prob_bytes() { return sizeof(GemmProb); }
void gemm_prob_fill(void* dst, int i, const double2* A, const double2* B, double2* C, int m, int n, int k, int lda,
                    int ldb, int ldc, double2 alpha, int accumulate) {
    ((GemmProb*)dst)[i] = GemmProb{A, B, C, m, n, k, lda, ldb, ldc, alpha, accumulate};
}
cudaError_t launch_zgemm_batched(const void* probs, int nprob, int max_m, int max_n, cudaStream_t st) {
    if (nprob == 0) return cudaSuccess;
    const int tiles = ((max_m + GB - 1) / GB) * ((max_n + GB - 1) / GB);
    count_launch();
    zgemm_batched_kernel<<<dim3(tiles, nprob), 256, 0, st>>>((const GemmProb*)probs);
    return cudaGetLastError();
}

size_t habc_sub_bytes() { return sizeof(HabcSub); }
void habc_sub_fill(void* dst, int i, long long koff, long long toff, int Lb, const int* bo, const int* len,
                   const long long* moff, const int* tin) {
    HabcSub s;
    s.koff = koff;
    s.toff = toff;
    s.Lb = Lb;
    for (int q = 0; q < 4; ++q) { s.bo[q] = bo[q]; s.len[q] = len[q]; s.moff[q] = moff[q]; s.tin[q] = tin[q]; }
    ((HabcSub*)dst)[i] = s;
}

template <typename T>
cudaError_t launch_habc_form(const void* subs, int nsub, int max_Lb, const T* K, const TraceCoef<double2>* tc,
                             double2* K64, const double2* KR, double2* W, int phase, cudaStream_t st) {
    const long long LL = (long long)max_Lb * max_Lb;
    const int bx = (int)std::min<long long>(1024, (LL + 255) / 256);
    count_launch();
    habc_form_kernel<T><<<dim3(bx, nsub), 256, 0, st>>>((const HabcSub*)subs, K, tc, K64, KR, W, phase);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_habc_final(const void* subs, int nsub, int max_Lb, const double2* Mside,
                              const TraceCoef<double2>* tc, const double2* P1, const double2* RP, const double2* W,
                              const double2* RW, T* Q, T* Lq, T* D1, T* D2, cudaStream_t st) {
    const long long LL = (long long)max_Lb * max_Lb;
    const int bx = (int)std::min<long long>(1024, (LL + 255) / 256);
    count_launch();
    habc_final_kernel<T><<<dim3(bx, nsub), 256, 0, st>>>((const HabcSub*)subs, Mside, tc, P1, RP, W, RW, Q, Lq, D1, D2);
    return cudaGetLastError();
}
template <typename T>
void launch_trace_swap(const T* in, T* out, const int* swp, long long ntrace, int nrhs, cudaStream_t st) {
    const long long tot = ntrace * nrhs;
    const int nb = (int)std::min<long long>(4096, (tot + 255) / 256);
    count_launch();
    trace_swap_kernel<T><<<nb, 256, 0, st>>>(in, out, swp, ntrace, nrhs);
}

template cudaError_t launch_habc_form<float2>(const void*, int, int, const float2*, const TraceCoef<double2>*, double2*,
                                              const double2*, double2*, int, cudaStream_t);
template cudaError_t launch_habc_form<double2>(const void*, int, int, const double2*, const TraceCoef<double2>*,
                                               double2*, const double2*, double2*, int, cudaStream_t);
template cudaError_t launch_habc_final<float2>(const void*, int, int, const double2*, const TraceCoef<double2>*,
                                               const double2*, const double2*, const double2*, const double2*, float2*,
                                               float2*, float2*, float2*, cudaStream_t);
template cudaError_t launch_habc_final<double2>(const void*, int, int, const double2*, const TraceCoef<double2>*,
                                                const double2*, const double2*, const double2*, const double2*,
                                                double2*, double2*, double2*, double2*, cudaStream_t);
template void launch_trace_swap<float2>(const float2*, float2*, const int*, long long, int, cudaStream_t);
template void launch_trace_swap<double2>(const double2*, double2*, const int*, long long, int, cudaStream_t);
