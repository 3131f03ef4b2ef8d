// Pair-symmetric FP32 pair sums: every unordered pair {i, j} is evaluated once
// and feeds both bodies.
//
// Forces (Section 2.3): the term of j on i is m_j s^-3/2 d and that of i on j
// is -m_i s^-3/2 d (d = x_j - x_i, s = |d|^2 + eps^2; Newton's third law), so
// the sum counted at 20 flops per ordered interaction in Section 4.1 costs 16
// FP32 lane operations per unordered pair, 8 per ordered interaction, against
// 12 in the one-sided kernel.
//
// Adjoint VJP (the reverse step's x-bar and m-bar sums; the one-sided
// VjpF32x2 policy states them): with f = s^-3/2, h = s^-5/2, e = abar_j . d,
// g = abar_i . d and c = m_j g - m_i e, body i gathers
//   U_i += f abar_j,  V_i += f m_j,  W_i += h c d,  P_i += f e
// and, from the same pair seen from j (d -> -d, e <-> -g, so c is unchanged),
//   U_j += f abar_i,  V_j += f m_i,  W_j -= h c d,  P_j -= f g;
// 34 lane operations per unordered pair (d, s, f, h, e, g, c shared) against
// 2 x 26 one-sided. The VJP's own pair (j == i) is masked: its f = eps^-3
// terms cancel only in the epilogue's FP32 sums.
//
// Precision form (FP64 state, Section 2.3's sum with compensated
// accumulation): the force pair terms in FP32, FP32 sums within a block pair,
// and the block-pair partials two-summed in the epilogue before the FP64
// update.
//
// Work decomposition. Bodies are padded with zero-mass bodies to nb blocks of
// B = 32 x W x R. An item is a block pair (bi, bj), bi <= bj, one CTA each.
// Each warp of the CTA owns 32 x R bodies of block bi, R per lane, held
// duplicated in f32x2 registers as in the one-sided kernels; block bj is
// walked in chunks of 32 records (64 bodies), one record per lane, and for
// 32 rounds every lane evaluates its R i-bodies against the two bodies of its
// current record, then passes the record and the record's running j-side sums
// to the next lane (shuffles). After 32 rounds each record is back home with
// its sums over the warp's i-bodies, which land in the warp's slice of shared
// memory; at the end the CTA adds the W slices in warp order. The diagonal
// item (bi == bj) evaluates every ordered pair of its block from the i side
// only.
//
// Determinism. The partial sums land in P[p][k][b] (p = the partner block: bj
// for the i side of item (bi, bj), bi for its j side; k = the sum), which
// every body fills exactly once for each p; a second kernel adds
// P[0..nb-1][k][b] in that order and runs the policy's epilogue, so the
// result does not depend on scheduling.
#include <cstring>

#include "kernels.h"

namespace nb {
namespace {

__device__ __forceinline__ float2 shfl2(float2 v, int src) {
    return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

// Forces.
#ifndef NB_SYM_ACCEL_REC_SMEM
#define NB_SYM_ACCEL_REC_SMEM 0  // records by shuffle: 3.987e12 against 3.962e12 staged (N = 262144)
#endif
#ifndef NB_SYM_VJP_REC_SMEM
#define NB_SYM_VJP_REC_SMEM 1  // records staged: 2.6 against 2.8 ms at N = 65536, 46.9 against 49.2 ms per C5 adjoint
#endif

struct SymAccel {
    static constexpr int R = kSymR;
    static constexpr bool REC_SMEM = NB_SYM_ACCEL_REC_SMEM;  // chunk records staged in shared memory
    static constexpr int REGS = 128;  // register target: 4 CTAs of 4 warps per SM (126 used)
    static constexpr int NACC = 3;      // a_x, a_y, a_z
    static constexpr int REC_F4 = 2;    // {x0,x1,y0,y1} {z0,z1,m0,m1}
    static constexpr bool SELF_MASK = false;  // d = 0 gives exactly 0
    static constexpr bool BLOCK_CALL = true;
    __host__ __device__ static constexpr float jsign(int) { return -1.f; }
    struct I { float2 nx, ny, nz, m; };
    struct J { float2 x, y, z, m; };
    struct C { float2 eps2; };
    __device__ static void consts(const ForceArgs &a, C &c) { c.eps2 = dup(a.eps2); }
    // Positions are read-only for the whole step (the step's epilogue writes
    // the other buffer). A tile launch other than the first of its step does
    // not wait for the grid that wrote them, but that grid completed before
    // the first tile's CTAs passed their wait and so before this launch
    // began.
    __device__ static void load_i(const ForceArgs &a, int64_t i, I &s) {
        s.nx = dup(-pair_get(a.src, i, 0));
        s.ny = dup(-pair_get(a.src, i, 1));
        s.nz = dup(-pair_get(a.src, i, 2));
        s.m = dup(pair_get(a.src, i, 3));
    }
    __device__ static void load_j(const float4 *rec, J &j) {
        const float4 r0 = __ldg(rec), r1 = __ldg(rec + 1);
        j.x = f2(r0.x, r0.y);
        j.y = f2(r0.z, r0.w);
        j.z = f2(r1.x, r1.y);
        j.m = f2(r1.z, r1.w);
    }
    __device__ static void shfl(J &j, int src) {
        j.x = shfl2(j.x, src);
        j.y = shfl2(j.y, src);
        j.z = shfl2(j.z, src);
        j.m = shfl2(j.m, src);
    }
    // record q of a chunk staged in shared memory as [REC_F4][32] float4
    __device__ static void load_j_smem(const float4 *rb, int q, J &j) {
        const float4 r0 = rb[q], r1 = rb[32 + q];
        j.x = f2(r0.x, r0.y);
        j.y = f2(r0.z, r0.w);
        j.z = f2(r1.x, r1.y);
        j.m = f2(r1.z, r1.w);
    }
    template <bool MASK>
    __device__ __forceinline__ static void pair(const J &j, const I &s, float2 (&ai)[NACC],
                                                float2 (&aj)[NACC], const C &c, float2) {
        const float2 dx = __fadd2_rn(j.x, s.nx);
        const float2 dy = __fadd2_rn(j.y, s.ny);
        const float2 dz = __fadd2_rn(j.z, s.nz);
        float2 q = __ffma2_rn(dx, dx, c.eps2);
        q = __ffma2_rn(dy, dy, q);
        q = __ffma2_rn(dz, dz, q);
        const float2 y = rsqrt_mufu2(q);
        const float2 y3 = __fmul2_rn(__fmul2_rn(y, y), y);
        const float2 wi = __fmul2_rn(j.m, y3);  // j on i: +m_j s^-3/2 d
        ai[0] = __ffma2_rn(wi, dx, ai[0]);
        ai[1] = __ffma2_rn(wi, dy, ai[1]);
        ai[2] = __ffma2_rn(wi, dz, ai[2]);
        const float2 wj = __fmul2_rn(s.m, y3);  // i on j: -m_i s^-3/2 d (sign at the store)
        aj[0] = __ffma2_rn(wj, dx, aj[0]);
        aj[1] = __ffma2_rn(wj, dy, aj[1]);
        aj[2] = __ffma2_rn(wj, dz, aj[2]);
    }
    // across partials: plain FP32 sums in block order
    static constexpr bool COMP = false;
    struct Fin { float s[NACC]; };
    __device__ static void fin_set(Fin &f, int k, float h, float) { f.s[k] = h; }
    __device__ static void finish(const ForceArgs &a, int64_t i, const Fin &f) {
        const float G = (float)a.G;
        finish_fp32(a, i, G * f.s[0], G * f.s[1], G * f.s[2]);
    }
};

// Precision form (FP64 state): the pair terms of SymAccel from the FP32
// packed positions; each block-pair partial is an FP32 sum, and the epilogue
// two-sums the partials in block order into (hi, lo) per component (about
// 2^-44 relative), widens once and runs the FP64 update, as the one-sided
// compensated policy does with its tile sums.
struct SymComp : SymAccel {
    static constexpr bool COMP = true;
    struct Fin { float h[NACC], l[NACC]; };
    __device__ static void fin_set(Fin &f, int k, float h, float l) {
        f.h[k] = h;
        f.l[k] = l;
    }
    __device__ static void finish(const ForceArgs &a, int64_t i, const Fin &f) {
        finish_fp64(a, i, a.G * ((double)f.h[0] + (double)f.l[0]), a.G * ((double)f.h[1] + (double)f.l[1]),
                    a.G * ((double)f.h[2] + (double)f.l[2]));
    }
};

// Adjoint VJP: sums (U_x, U_y, U_z, V, W_x, W_y, W_z, P), records as the
// one-sided VJP's {x0,x1,y0,y1} {z0,z1,m0,m1} {ax0,ax1,ay0,ay1} {az0,az1,0,0}.
#ifndef NB_SYM_VJP_REGS
#define NB_SYM_VJP_REGS 168  // 3 CTAs of 4 warps per SM; 128 (4 CTAs) spills: 52.3 against 49.2 ms for the N = 16384 adjoint
#endif
struct SymVjp {
    static constexpr int R = kSymVjpR;
    static constexpr bool REC_SMEM = NB_SYM_VJP_REC_SMEM;
    static constexpr int REGS = NB_SYM_VJP_REGS;  // register target
    static constexpr int NACC = 8;
    static constexpr int REC_F4 = 4;
    static constexpr bool SELF_MASK = true;
    static constexpr bool BLOCK_CALL = false;
    // j side: U as is; V gathered with -m_i; W and P with the sign flipped
    __host__ __device__ static constexpr float jsign(int k) { return k < 3 ? 1.f : -1.f; }
    struct I { float2 nx, ny, nz, nm, ax, ay, az; };  // nm = -m_i
    struct J { float2 x, y, z, m, ax, ay, az; };
    struct C { float2 eps2; };
    __device__ static void consts(const ForceArgs &a, C &c) { c.eps2 = dup(a.eps2); }
    __device__ static void load_i(const ForceArgs &a, int64_t i, I &s) {
        s.nx = dup(-vrec_get(a.src, i, 0));
        s.ny = dup(-vrec_get(a.src, i, 1));
        s.nz = dup(-vrec_get(a.src, i, 2));
        s.nm = dup(-vrec_get(a.src, i, 3));
        s.ax = dup(vrec_get(a.src, i, 4));
        s.ay = dup(vrec_get(a.src, i, 5));
        s.az = dup(vrec_get(a.src, i, 6));
    }
    __device__ static void load_j(const float4 *rec, J &j) {
        const float4 r0 = __ldg(rec), r1 = __ldg(rec + 1), r2 = __ldg(rec + 2), r3 = __ldg(rec + 3);
        j.x = f2(r0.x, r0.y);
        j.y = f2(r0.z, r0.w);
        j.z = f2(r1.x, r1.y);
        j.m = f2(r1.z, r1.w);
        j.ax = f2(r2.x, r2.y);
        j.ay = f2(r2.z, r2.w);
        j.az = f2(r3.x, r3.y);
    }
    __device__ static void shfl(J &j, int src) {
        j.x = shfl2(j.x, src);
        j.y = shfl2(j.y, src);
        j.z = shfl2(j.z, src);
        j.m = shfl2(j.m, src);
        j.ax = shfl2(j.ax, src);
        j.ay = shfl2(j.ay, src);
        j.az = shfl2(j.az, src);
    }
    __device__ static void load_j_smem(const float4 *rb, int q, J &j) {
        const float4 r0 = rb[q], r1 = rb[32 + q], r2 = rb[64 + q];
        const float2 r3 = *reinterpret_cast<const float2 *>(rb + 96 + q);
        j.x = f2(r0.x, r0.y);
        j.y = f2(r0.z, r0.w);
        j.z = f2(r1.x, r1.y);
        j.m = f2(r1.z, r1.w);
        j.ax = f2(r2.x, r2.y);
        j.ay = f2(r2.z, r2.w);
        j.az = r3;
    }
    template <bool MASK>
    __device__ __forceinline__ static void pair(const J &j, const I &s, float2 (&ai)[NACC],
                                                float2 (&aj)[NACC], const C &c, float2 keep) {
        terms<MASK>(__fadd2_rn(j.x, s.nx), __fadd2_rn(j.y, s.ny), __fadd2_rn(j.z, s.nz), j, s, ai, aj,
                    c, keep);
    }
    // The pair's terms for both bodies from the separation d = x_j - x_i.
    template <bool MASK>
    __device__ __forceinline__ static void terms(float2 dx, float2 dy, float2 dz, const J &j, const I &s,
                                                 float2 (&ai)[NACC], float2 (&aj)[NACC], const C &c,
                                                 float2 keep) {
        float2 q = __ffma2_rn(dx, dx, c.eps2);
        q = __ffma2_rn(dy, dy, q);
        q = __ffma2_rn(dz, dz, q);
        float2 y = rsqrt_mufu2(q);
        if constexpr (MASK) y = __fmul2_rn(y, keep);
        const float2 y2 = __fmul2_rn(y, y);
        const float2 f = __fmul2_rn(y, y2);
        const float2 h = __fmul2_rn(f, y2);
        float2 e = __fmul2_rn(j.ax, dx);  // abar_j . d
        e = __ffma2_rn(j.ay, dy, e);
        e = __ffma2_rn(j.az, dz, e);
        float2 g = __fmul2_rn(s.ax, dx);  // abar_i . d
        g = __ffma2_rn(s.ay, dy, g);
        g = __ffma2_rn(s.az, dz, g);
        const float2 hc = __fmul2_rn(h, __ffma2_rn(j.m, g, __fmul2_rn(s.nm, e)));  // h (m_j g - m_i e)
        ai[0] = __ffma2_rn(f, j.ax, ai[0]);
        ai[1] = __ffma2_rn(f, j.ay, ai[1]);
        ai[2] = __ffma2_rn(f, j.az, ai[2]);
        ai[3] = __ffma2_rn(f, j.m, ai[3]);
        ai[4] = __ffma2_rn(hc, dx, ai[4]);
        ai[5] = __ffma2_rn(hc, dy, ai[5]);
        ai[6] = __ffma2_rn(hc, dz, ai[6]);
        ai[7] = __ffma2_rn(f, e, ai[7]);
        aj[0] = __ffma2_rn(f, s.ax, aj[0]);
        aj[1] = __ffma2_rn(f, s.ay, aj[1]);
        aj[2] = __ffma2_rn(f, s.az, aj[2]);
        aj[3] = __ffma2_rn(f, s.nm, aj[3]);
        aj[4] = __ffma2_rn(hc, dx, aj[4]);
        aj[5] = __ffma2_rn(hc, dy, aj[5]);
        aj[6] = __ffma2_rn(hc, dz, aj[6]);
        aj[7] = __ffma2_rn(f, g, aj[7]);
    }
    static constexpr bool COMP = false;
    struct Fin { float s[NACC]; };
    __device__ static void fin_set(Fin &f, int k, float h, float) { f.s[k] = h; }
    __device__ static void finish(const ForceArgs &a, int64_t k, const Fin &fin) {
        const float *s = fin.s;
        VjpF32x2::F f;
        f.ux = s[0]; f.uy = s[1]; f.uz = s[2]; f.v = s[3];
        f.wx = s[4]; f.wy = s[5]; f.wz = s[6]; f.p = s[7];
        VjpF32x2::finish(a, k, f);
    }
};

// Precision form of the VJP (FP64 state): the records of the one-sided
// VjpComp policy, {x0,x1,y0,y1} {z0,z1,m0,m1} {ax0,ax1,ay0,ay1}
// {az0,az1,xl0,xl1} {yl0,yl1,zl0,zl1} (the FP32 low parts of the FP64
// positions), d formed as (x_j^hi - x_i^hi) + (x_j^lo - x_i^lo) so that it
// keeps FP32 relative accuracy for close pairs (whose terms weigh as
// |d|^-3 ... |d|^-5), the pair terms of SymVjp, FP32 sums within a block
// pair, and the block-pair partials two-summed in the epilogue, which widens
// them and updates x-bar and m-bar in FP64 as the one-sided policy does.
#ifndef NB_SYM_VJP_COMP_REGS
#define NB_SYM_VJP_COMP_REGS 168
#endif
struct SymVjpComp {
    static constexpr int R = kSymVjpR;
    static constexpr bool REC_SMEM = NB_SYM_VJP_REC_SMEM;
    static constexpr int REGS = NB_SYM_VJP_COMP_REGS;
    static constexpr int NACC = 8;
    static constexpr int REC_F4 = 5;
    static constexpr bool SELF_MASK = true;
    static constexpr bool BLOCK_CALL = false;
    __host__ __device__ static constexpr float jsign(int k) { return SymVjp::jsign(k); }
    struct I {
        SymVjp::I b;
        float2 nlx, nly, nlz;
    };
    struct J {
        SymVjp::J b;
        float2 xl, yl, zl;
    };
    using C = SymVjp::C;
    __device__ static void consts(const ForceArgs &a, C &c) { SymVjp::consts(a, c); }
    __device__ static float get(const float4 *base, int64_t i, int c) {
        const float *p = reinterpret_cast<const float *>(base + (i >> 1) * 5);
        return p[2 * c + (int)(i & 1)];
    }
    __device__ static void load_i(const ForceArgs &a, int64_t i, I &s) {
        s.b.nx = dup(-get(a.src, i, 0));
        s.b.ny = dup(-get(a.src, i, 1));
        s.b.nz = dup(-get(a.src, i, 2));
        s.b.nm = dup(-get(a.src, i, 3));
        s.b.ax = dup(get(a.src, i, 4));
        s.b.ay = dup(get(a.src, i, 5));
        s.b.az = dup(get(a.src, i, 6));
        s.nlx = dup(-get(a.src, i, 7));
        s.nly = dup(-get(a.src, i, 8));
        s.nlz = dup(-get(a.src, i, 9));
    }
    __device__ static void from_f4(const float4 &r0, const float4 &r1, const float4 &r2, const float4 &r3,
                                   const float4 &r4, J &j) {
        j.b.x = f2(r0.x, r0.y);
        j.b.y = f2(r0.z, r0.w);
        j.b.z = f2(r1.x, r1.y);
        j.b.m = f2(r1.z, r1.w);
        j.b.ax = f2(r2.x, r2.y);
        j.b.ay = f2(r2.z, r2.w);
        j.b.az = f2(r3.x, r3.y);
        j.xl = f2(r3.z, r3.w);
        j.yl = f2(r4.x, r4.y);
        j.zl = f2(r4.z, r4.w);
    }
    __device__ static void load_j(const float4 *rec, J &j) {
        from_f4(__ldg(rec), __ldg(rec + 1), __ldg(rec + 2), __ldg(rec + 3), __ldg(rec + 4), j);
    }
    __device__ static void shfl(J &j, int src) {
        SymVjp::shfl(j.b, src);
        j.xl = shfl2(j.xl, src);
        j.yl = shfl2(j.yl, src);
        j.zl = shfl2(j.zl, src);
    }
    __device__ static void load_j_smem(const float4 *rb, int q, J &j) {
        from_f4(rb[q], rb[32 + q], rb[64 + q], rb[96 + q], rb[128 + q], j);
    }
    template <bool MASK>
    __device__ __forceinline__ static void pair(const J &j, const I &s, float2 (&ai)[NACC],
                                                float2 (&aj)[NACC], const C &c, float2 keep) {
        const float2 dx = __fadd2_rn(__fadd2_rn(j.b.x, s.b.nx), __fadd2_rn(j.xl, s.nlx));
        const float2 dy = __fadd2_rn(__fadd2_rn(j.b.y, s.b.ny), __fadd2_rn(j.yl, s.nly));
        const float2 dz = __fadd2_rn(__fadd2_rn(j.b.z, s.b.nz), __fadd2_rn(j.zl, s.nlz));
        SymVjp::terms<MASK>(dx, dy, dz, j.b, s.b, ai, aj, c, keep);
    }
    static constexpr bool COMP = true;
    struct Fin { float h[NACC], l[NACC]; };
    __device__ static void fin_set(Fin &f, int k, float h, float l) {
        f.h[k] = h;
        f.l[k] = l;
    }
    __device__ static void finish(const ForceArgs &a, int64_t k, const Fin &fin) {
        VjpComp::F f;
#pragma unroll
        for (int q = 0; q < NACC; ++q) {
            f.h[q] = fin.h[q];
            f.l[q] = fin.l[q];
        }
        VjpComp::finish(a, k, f);
    }
};

// Item t of the upper triangle of block pairs. With NB_SYM_DIAG_LAST the
// nb(nb-1)/2 off-diagonal pairs come first (row-major, bi < bj) and the nb
// diagonal items last: a diagonal item evaluates its block from one side
// only (about 3/4 of an off-diagonal item's operations), so the cheaper items
// fill the launch's last wave (measured at N = 262144: 3.987e12 against
// 3.932e12 interactions/s with each row starting with its diagonal item).
// Otherwise rows bi = 0..nb-1 hold bj = bi..nb-1. The order of the items
// changes no result: every partial has its own slot.
#ifndef NB_SYM_DIAG_LAST
#define NB_SYM_DIAG_LAST 1
#endif
__device__ __forceinline__ void sym_item(int t, int nb, int &bi, int &bj) {
    if constexpr (NB_SYM_DIAG_LAST) {
        const int off = nb * (nb - 1) / 2;
        if (t >= off) {
            bi = bj = t - off;
            return;
        }
        int r, c;
        tri_item(t, nb - 1, r, c);  // (r, c), c >= r, of nb - 1 columns: the pair (r, c + 1)
        bi = r;
        bj = c + 1;
        return;
    }
    tri_item(t, nb, bi, bj);
}

// The 32 rounds of one chunk. MASK: the diagonal item of a policy that
// masks its own pair; i_base (this lane's first i-body) and j_base (the
// chunk's first j-body) are offsets within the block.
#ifndef NB_SYM_ROUND_UNROLL
#define NB_SYM_ROUND_UNROLL 1  // two rounds per unrolled step measured within noise
#endif
constexpr int kRoundUnroll = NB_SYM_ROUND_UNROLL;  // rounds per unrolled step (build flag)

template <class S, bool MASK>
__device__ __forceinline__ void chunk_rounds(typename S::J &sj, const typename S::I (&si)[S::R],
                                             float2 (&ai)[S::R][S::NACC], float2 (&aj)[S::NACC],
                                             const typename S::C &c, int l, int next, int i_base,
                                             int j_base) {
#pragma unroll kRoundUnroll
    for (int round = 0; round < 32; ++round) {
        const int j0 = j_base + 2 * ((l + round) & 31);  // the current record's first body
#pragma unroll
        for (int r = 0; r < S::R; ++r) {
            float2 keep = f2(1.f, 1.f);
            if constexpr (MASK) {
                const int i = i_base + 32 * r;
                keep = f2(i == j0 ? 0.f : 1.f, i == j0 + 1 ? 0.f : 1.f);
            }
            S::template pair<MASK>(sj, si[r], ai[r], aj, c, keep);
        }
        S::shfl(sj, next);
#pragma unroll
        for (int k = 0; k < S::NACC; ++k) aj[k] = shfl2(aj[k], next);
    }
}

// The same 32 rounds with the chunk's records staged in shared memory
// (rb: [REC_F4][32] float4): at round r lane l reads record (l + r) mod 32
// itself, so only the running j-side sums travel between lanes.
template <class S, bool MASK>
__device__ __forceinline__ void chunk_rounds_smem(const float4 *rb, const typename S::I (&si)[S::R],
                                                  float2 (&ai)[S::R][S::NACC], float2 (&aj)[S::NACC],
                                                  const typename S::C &c, int l, int next, int i_base,
                                                  int j_base) {
#pragma unroll kRoundUnroll
    for (int round = 0; round < 32; ++round) {
        const int q = (l + round) & 31;
        const int j0 = j_base + 2 * q;
        typename S::J sj;
        S::load_j_smem(rb, q, sj);
#pragma unroll
        for (int r = 0; r < S::R; ++r) {
            float2 keep = f2(1.f, 1.f);
            if constexpr (MASK) {
                const int i = i_base + 32 * r;
                keep = f2(i == j0 ? 0.f : 1.f, i == j0 + 1 ? 0.f : 1.f);
            }
            S::template pair<MASK>(sj, si[r], ai[r], aj, c, keep);
        }
#pragma unroll
        for (int k = 0; k < S::NACC; ++k) aj[k] = shfl2(aj[k], next);
    }
}

// Tiled launches: the partials of one tile, [slot][side][k][b] (slot = the
// block pair's index in its tile, side 0 = the i side for block bi, 1 = the
// j side for block bj, b = body within the block), and the partner range of
// a block in a tile. tile_partners returns the number of partner blocks of
// block `beta` in tile g (0 if the tile does not touch it) and sets the
// first one; partner p's partial is on side 1 (p < beta: the j side of item
// (p, beta)) at slot tile_slot(g, p, beta), else on side 0 at
// tile_slot(g, beta, p).
__device__ __forceinline__ int tile_partners(const SymTile &g, int beta, int &p0) {
    if (beta >= g.c0 && beta < g.c0 + g.hc) {  // column strip (and the diagonal tile's strip)
        p0 = g.r0;
        return g.hr;
    }
    if (g.I != g.J && beta >= g.r0 && beta < g.r0 + g.hr) {  // row strip
        p0 = g.c0;
        return g.hc;
    }
    p0 = 0;
    return 0;
}
__device__ __forceinline__ int tile_slot(const SymTile &g, int bi, int bj) {
    if (g.I == g.J) {
        const int r = bi - g.r0, c = bj - g.r0;
        return r * g.hr - r * (r - 1) / 2 + (c - r);
    }
    return (bi - g.r0) * g.hc + (bj - g.c0);
}

// Add tile g's partials of body `o` of block `beta`, all NA sums, to the
// running sums (hi, lo) in partner order; the tile whose first partner is
// block 0 starts them. FP32 sums, or two-sums in the precision form, as the
// one-launch epilogue adds its partials.
template <class S, int B>
__device__ __forceinline__ void tile_fold_body(const ForceArgs &a, const float *acc, const float *buf,
                                               const SymTile &g, int beta, int o, float (&h)[S::NACC],
                                               float (&l)[S::NACC]) {
    constexpr int NA = S::NACC;
    int p0;
    const int np = tile_partners(g, beta, p0);
    const int64_t b = (int64_t)beta * B + o;
    if (p0 == 0) {
#pragma unroll
        for (int k = 0; k < NA; ++k) h[k] = l[k] = 0.f;
    } else {
#pragma unroll
        for (int k = 0; k < NA; ++k) {
            h[k] = __ldcg(acc + (int64_t)k * a.npad + b);
            l[k] = S::COMP ? __ldcg(acc + (int64_t)(NA + k) * a.npad + b) : 0.f;
        }
    }
    // partners in batches: the batch's loads are issued together, then
    // added in partner order
    constexpr int PB = NA <= 4 ? 8 : 4;
    for (int q0 = 0; q0 < np; q0 += PB) {
        float v[PB][NA];
#pragma unroll
        for (int j = 0; j < PB; ++j) {
            const int p = p0 + q0 + j;
            if (q0 + j < np) {
                const int side = p < beta ? 1 : 0;
                const int slot = side ? tile_slot(g, p, beta) : tile_slot(g, beta, p);
                const float *src = buf + ((int64_t)(slot * 2 + side) * NA) * B + o;
#pragma unroll
                for (int k = 0; k < NA; ++k) v[j][k] = __ldcs(src + k * B);
            }
        }
#pragma unroll
        for (int j = 0; j < PB; ++j) {
            if (q0 + j >= np) break;
#pragma unroll
            for (int k = 0; k < NA; ++k) {
                if constexpr (S::COMP) {
                    float sum, e;
                    two_sum(h[k], v[j][k], sum, e);
                    h[k] = sum;
                    l[k] = __fadd_rn(l[k], e);
                } else {
                    h[k] += v[j][k];
                }
            }
        }
    }
}

// Floats of one tile buffer: w x w slots of 2 sides x NA sums x B bodies.
// `part` holds two of them (tiles alternate), then the running sums
// [2][NA][npad].
template <class S, int B>
__host__ __device__ constexpr int64_t tile_buf_floats(int w) {
    return (int64_t)w * w * 2 * S::NACC * B;
}

// Threads per CTA: W i-warps, each with JS warps that hold the same i-bodies
// and split the block pair's j-chunks between them (JS > 1: the forces).
template <int W, int JS>
__host__ __device__ constexpr int sym_threads() {
    return W * 32 * JS;
}

// Fold the previous tile into the running sums: units of one body per
// thread of the blocks it touched (its row strip, then its column strip),
// spread over this launch's CTAs. Not inlined: the pair loop before
// the call keeps all the registers (inlined, this code cost the loop 2.6 %
// at N = 262144 without ever running).
template <class S, int W, int JS>
__device__ __noinline__ void tile_fold_prev(const ForceArgs &a) {
    constexpr int R = S::R, B = W * 32 * R, NA = S::NACC;
    const int nb = (int)(a.npad / B);
    float *P = reinterpret_cast<float *>(a.part);
    const SymTile pg = sym_tile(a.tile - 1, nb, a.tile_w);
    const float *pbuf = P + ((a.tile - 1) & 1) * tile_buf_floats<S, B>(a.tile_w);
    float *acc = P + 2 * tile_buf_floats<S, B>(a.tile_w);
    const int nblk = pg.I == pg.J ? pg.hr : pg.hr + pg.hc;
    constexpr int NT = sym_threads<W, JS>();
    constexpr int kUnits = B / NT;  // units per block
    for (int u = blockIdx.x; u < nblk * kUnits; u += gridDim.x) {
        const int kb = u / kUnits;
        const int beta = kb < pg.hr ? pg.r0 + kb : pg.c0 + (kb - pg.hr);
        const int o = (u % kUnits) * NT + threadIdx.x;
        float h[NA], lo[NA];
        tile_fold_body<S, B>(a, acc, pbuf, pg, beta, o, h, lo);
        const int64_t b = (int64_t)beta * B + o;
#pragma unroll
        for (int k = 0; k < NA; ++k) {
            __stcg(acc + (int64_t)k * a.npad + b, h[k]);
            if (S::COMP) __stcg(acc + (int64_t)(NA + k) * a.npad + b, lo[k]);
        }
    }
}

// Resident CTAs per SM that keep a policy's registers at its target (the
// compiler's own choice without a bound; a bound of 1 CTA let it take 210 for
// the VJP).
template <class S, int W, int JS = 1>
__host__ __device__ constexpr int sym_min_blocks() {
    return 65536 / (sym_threads<W, JS>() * S::REGS) > 0 ? 65536 / (sym_threads<W, JS>() * S::REGS) : 1;
}

// Record buffers per warp of the staged-record kernels: two unless the
// second would lower the resident CTAs per SM below what the registers allow
// (228 KiB of shared memory per SM; the VJP's 512-body blocks: 3 CTAs of 81
// KiB do not fit, of 73 KiB they do).
template <class S, int W>
__host__ __device__ constexpr int rec_bufs() {
    constexpr size_t base = (size_t)W * S::NACC * (W * 32 * S::R) * 4;
    constexpr size_t buf = (size_t)W * S::REC_F4 * 32 * 16;
    // (1 KiB of each CTA's shared memory is reserved by the system)
    return (base + 2 * buf + 1024) * sym_min_blocks<S, W>() <= (size_t)228 * 1024 ? 2 : 1;
}


// The pair work of block pair (bi, bj) and its partials: the i side's NA sums
// of the bodies of block bi to pi[k * ps + o] and the j side's of block bj to
// pj[k * ps + o] (o = the body's offset in its block). late_wait: wait for
// the previous grid before the first write (tile launches). For the forces
// (S::BLOCK_CALL) the two kernels call it out of line, so that the one-launch
// and the tile kernels run the same compiled pair loop: inlined into each,
// the tile kernel's copy ran 0.8 % slower (3.94e12 against 3.99e12
// interactions/s at N = 262144 with tiles of 24 to 96 blocks, 3.97e12
// against 4.02e12 for the precision form at N = 2^20). The VJPs' one-launch
// kernel keeps it inlined (out of line, the N = 16384 adjoint took 47.0
// against 46.8 ms) and their tile kernel calls it out of line (10.07 ms per
// VJP at N = 131072 by tiles of 20 blocks, against 10.15 inlined and 10.10
// in one launch). JS > 1 (the forces' split 256-body blocks): JS warps hold
// the same i-bodies and each walks its C of the block pair's chunks, so a
// chunk's j-side sums come from one warp, and the i-side sums of the warps
// are added in warp order through shared memory before the one store (at
// N = 16384, 83.7 against 94-95 us per FP32 step with one warp per block
// pair: where the block pairs are few, the SMs hold more warps).
template <class S, int W, int JS>
__device__ __forceinline__ void sym_block_body(const ForceArgs &a, int bi, int bj, float *pi, float *pj,
                                               int64_t ps, bool late_wait) {
    constexpr int R = S::R, B = W * 32 * R, NA = S::NACC;
    constexpr int NT = sym_threads<W, JS>(), C = B / 64 / JS;  // chunks per warp
    static_assert(!(S::REC_SMEM && JS > 1), "split j-chunks with records by shuffle only");
    extern __shared__ float acc_j[];  // [W][NA][B], then with JS > 1 [JS - 1][R][NA][32]
    const int w = JS > 1 ? (threadIdx.x >> 5) % W : threadIdx.x >> 5;  // the i-warp
    const int js = JS > 1 ? (threadIdx.x >> 5) / W : 0;                 // its share of the chunks
    const int l = threadIdx.x & 31;
    const int next = (l + 1) & 31;
    typename S::C c;
    S::consts(a, c);
    typename S::I si[R];
    float2 ai[R][NA];
    const int i_base = w * 32 * R + l;  // offset of this lane's first i-body in block bi
    const int64_t gbase = (int64_t)bi * B;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        S::load_i(a, gbase + i_base + 32 * r, si[r]);
#pragma unroll
        for (int k = 0; k < NA; ++k) ai[r][k] = f2(0.f, 0.f);
    }
    const bool diag = bi == bj;
    float *mine = acc_j + w * NA * B;
    // S::REC_SMEM: this warp's record buffers after acc_j, [NBUF][REC_F4][32]
    // float4. With two, chunk ch + 1 is copied while chunk ch is evaluated;
    // with one (where two would cost a resident CTA per SM), each chunk's copy
    // is waited for at its start.
    constexpr int NBUF = rec_bufs<S, W>();
    float4 *rbw = reinterpret_cast<float4 *>(acc_j + W * NA * B) + w * NBUF * S::REC_F4 * 32;
    auto issue = [&](int ch) {
        const float4 *src = a.src + ((int64_t)bj * (B / 2) + ch * 32 + l) * S::REC_F4;
        float4 *dst = rbw + (ch % NBUF) * S::REC_F4 * 32 + l;
#pragma unroll
        for (int f = 0; f < S::REC_F4; ++f) cp_async16(dst + f * 32, src + f);
        cp_async_commit();
    };
    if constexpr (S::REC_SMEM && NBUF == 2) issue(0);
    for (int ch = js * C; ch < (js + 1) * C; ++ch) {
        float2 aj[NA];
#pragma unroll
        for (int k = 0; k < NA; ++k) aj[k] = f2(0.f, 0.f);
        if constexpr (S::REC_SMEM) {
            if constexpr (NBUF == 2) {
                if (ch + 1 < B / 64)
                    issue(ch + 1);
                else
                    cp_async_commit();  // an empty group keeps "all but the newest" meaning chunk ch
                cp_async_wait<1>();
            } else {
                issue(ch);
                cp_async_wait<0>();
            }
            __syncwarp();
            const float4 *rb = rbw + (ch % NBUF) * S::REC_F4 * 32;
            if (S::SELF_MASK && diag)
                chunk_rounds_smem<S, true>(rb, si, ai, aj, c, l, next, i_base, ch * 64);
            else
                chunk_rounds_smem<S, false>(rb, si, ai, aj, c, l, next, i_base, ch * 64);
            __syncwarp();  // every lane is done with the buffer before it is refilled
        } else {
            const int64_t q = (int64_t)bj * (B / 2) + ch * 32 + l;  // this lane's record
            typename S::J sj;
            S::load_j(a.src + q * S::REC_F4, sj);
            if (S::SELF_MASK && diag)
                chunk_rounds<S, true>(sj, si, ai, aj, c, l, next, i_base, ch * 64);
            else
                chunk_rounds<S, false>(sj, si, ai, aj, c, l, next, i_base, ch * 64);
        }
        if (!diag) {
            const int kb = ch * 64 + 2 * l;
#pragma unroll
            for (int k = 0; k < NA; ++k) {
                mine[k * B + kb] = S::jsign(k) * aj[k].x;
                mine[k * B + kb + 1] = S::jsign(k) * aj[k].y;
            }
        }
    }
    if (late_wait) asm volatile("griddepcontrol.wait;" ::: "memory");
    if constexpr (JS > 1) {
        // the i side: the j-split warps' sums of the same bodies, added in
        // warp order by the first
        float *xs = acc_j + W * NA * B;
        if (js > 0) {
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int k = 0; k < NA; ++k) xs[(((js - 1) * R + r) * NA + k) * 32 + l] = ai[r][k].x + ai[r][k].y;
        }
        __syncthreads();
        if (js == 0) {
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int k = 0; k < NA; ++k) {
                    float v = ai[r][k].x + ai[r][k].y;
#pragma unroll
                    for (int q = 1; q < JS; ++q) v += xs[(((q - 1) * R + r) * NA + k) * 32 + l];
                    __stcg(pi + k * ps + i_base + 32 * r, v);
                }
        }
    } else {
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int k = 0; k < NA; ++k) __stcg(pi + k * ps + i_base + 32 * r, ai[r][k].x + ai[r][k].y);
    }
    if (!diag) {
        __syncthreads();
        for (int t = threadIdx.x; t < B; t += NT) {
#pragma unroll
            for (int k = 0; k < NA; ++k) {
                float s = 0.f;
#pragma unroll
                for (int u = 0; u < W; ++u) s += acc_j[(u * NA + k) * B + t];
                __stcg(pj + k * ps + t, s);
            }
        }
    }
}

template <class S, int W, int JS>
__device__ __noinline__ void sym_block_call(const ForceArgs &a, int bi, int bj, float *pi, float *pj, int64_t ps,
                                            bool late_wait) {
    sym_block_body<S, W, JS>(a, bi, bj, pi, pj, ps, late_wait);
}
template <class S, int W, int JS, bool TILED>
__device__ __forceinline__ void sym_block(const ForceArgs &a, int bi, int bj, float *pi, float *pj, int64_t ps,
                                          bool late_wait) {
    if constexpr (S::BLOCK_CALL || TILED)
        sym_block_call<S, W, JS>(a, bi, bj, pi, pj, ps, late_wait);
    else
        sym_block_body<S, W, JS>(a, bi, bj, pi, pj, ps, late_wait);
}

// TILED: one launch per tile (the launch's tile and its fold of the previous
// tile); otherwise one launch over every block pair. Both run sym_block.
template <class S, int W, int JS, bool TILED>
__global__ void __launch_bounds__(sym_threads<W, JS>(), (sym_min_blocks<S, W, JS>())) sym_kernel(const ForceArgs a) {
    constexpr int R = S::R, B = W * 32 * R, NA = S::NACC;
    // the previous step's epilogue (it reads the partials and writes the
    // records read here) must be complete: the first (or only) launch of a
    // step waits for it; a later tile launch starts early, its records
    // written before the step's first tile began, and waits in sym_block
    // before it writes partials
    if (!TILED || a.tile == 0) asm volatile("griddepcontrol.wait;" ::: "memory");
    // tiles: the next tile's CTAs may take the SMs this launch's last wave
    // leaves (each waits for this grid before writing anything)
    if constexpr (TILED) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int nb = (int)(a.npad / B);
    float *P = reinterpret_cast<float *>(a.part);
    int bi, bj;
    if constexpr (TILED) {
        const SymTile g = sym_tile(a.tile, nb, a.tile_w);
        if (g.I == g.J) {
            int r, cc;
            tri_item(blockIdx.x, g.hr, r, cc);
            bi = g.r0 + r;
            bj = g.r0 + cc;
        } else {
            bi = g.r0 + (int)(blockIdx.x / g.hc);
            bj = g.c0 + (int)(blockIdx.x % g.hc);
        }
        // this item's slot of the tile buffer: [side][k][b], side 0 for block bi
        float *pi = P + (a.tile & 1) * tile_buf_floats<S, B>(a.tile_w) + ((int64_t)blockIdx.x * 2) * NA * B;
        sym_block<S, W, JS, true>(a, bi, bj, pi, pi + NA * B, B, true);
        // the previous tile's grid is complete (waited for in sym_block): its
        // partials are final for the fold, and this buffer (the tile before
        // it) is folded
        if (a.tile > 0) tile_fold_prev<S, W, JS>(a);
    } else {
        sym_item(blockIdx.x, nb, bi, bj);
        const int64_t np = a.npad;
        // P[p][k][b]: row bj for block bi's bodies, row bi for block bj's
        sym_block<S, W, JS, false>(a, bi, bj, P + (int64_t)bj * NA * np + (int64_t)bi * B,
                        P + (int64_t)bi * NA * np + (int64_t)bj * B, np, false);
        asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    }
}

// Sum of the nb partials of each body in block order (the policy's Fin:
// plain FP32, or two-sums in the precision form), then the policy's epilogue.
// A CTA takes 32 bodies with one warp per sum: lane l of warp k adds sum k of
// body l over the partner blocks (coalesced rows, every warp's loads in
// flight together), the warps meet in shared memory, and warp 0 runs the
// epilogue of its 32 bodies. (One thread per body walked its partials one
// round trip at a time: 43 us per VJP launch at N = 16384 against the pair
// kernel's 180 us; 103 against 100 us per forward step.)
template <class S>
__global__ void __launch_bounds__(32 * S::NACC) sym_finish_kernel(const ForceArgs a) {
    constexpr int NA = S::NACC;
    __shared__ float sh[NA][32], sl[NA][32];
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int lane = threadIdx.x & 31, k = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * 32 + lane;
    float h = 0.f, l = 0.f;
    if (i < a.n) {
        const float *q = reinterpret_cast<const float *>(a.part) + (int64_t)k * a.npad + i;
        const int64_t stride = (int64_t)NA * a.npad;  // one partner block
#pragma unroll 16
        for (int p = 0; p < a.ntiles; ++p) {
            const float v = __ldcs(q + p * stride);
            if constexpr (S::COMP) {
                float sum, e;
                two_sum(h, v, sum, e);
                h = sum;
                l = __fadd_rn(l, e);
            } else {
                h += v;
            }
        }
    }
    sh[k][lane] = h;
    sl[k][lane] = l;
    __syncthreads();
    if (k == 0 && i < a.n) {
        typename S::Fin f;
#pragma unroll
        for (int c = 0; c < NA; ++c) S::fin_set(f, c, sh[c][lane], sl[c][lane]);
        S::finish(a, i, f);
    }
    // No early trigger: the next step's pair kernel is scheduled when this
    // grid completes, onto all SMs at once. Triggered here, its few hundred
    // CTAs took the SMs as this grid's CTAs left them and piled onto some:
    // 182 against 100 us per step at N = 16384 (measured).
}

// After the last tile: its partials folded into the running sums of the
// bodies it touches, then the policy's epilogue for every body (one thread
// per body; the sums of every other body are complete in `acc`).
template <class S, int B>
__global__ void __launch_bounds__(128) sym_tile_final_kernel(const ForceArgs a) {
    constexpr int NA = S::NACC;
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const int nb = (int)(a.npad / B);
    const SymTile g = sym_tile(a.ntile - 1, nb, a.tile_w);
    const int beta = (int)(i / B), o = (int)(i % B);
    const float *P = reinterpret_cast<const float *>(a.part);
    const float *acc = P + 2 * tile_buf_floats<S, B>(a.tile_w);
    float h[NA], l[NA];
    int p0;
    if (tile_partners(g, beta, p0) > 0) {
        tile_fold_body<S, B>(a, acc, P + ((a.ntile - 1) & 1) * tile_buf_floats<S, B>(a.tile_w), g, beta, o,
                             h, l);
    } else {
#pragma unroll
        for (int k = 0; k < NA; ++k) {
            h[k] = __ldcg(acc + (int64_t)k * a.npad + i);
            l[k] = S::COMP ? __ldcg(acc + (int64_t)(NA + k) * a.npad + i) : 0.f;
        }
    }
    typename S::Fin f;
#pragma unroll
    for (int k = 0; k < NA; ++k) S::fin_set(f, k, h[k], l[k]);
    S::finish(a, i, f);
}

cudaError_t launch_ex(const void *fn, dim3 grid, dim3 block, size_t smem, bool pdl,
                      const ForceArgs &a, cudaStream_t st) {
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof cfg);
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    void *args[] = {const_cast<ForceArgs *>(&a)};
    return cudaLaunchKernelExC(&cfg, fn, args);
}

template <class S, int W, int JS>
constexpr size_t sym_smem() {
    return (size_t)W * S::NACC * (W * 32 * S::R) * 4 +
           (size_t)(JS - 1) * S::R * S::NACC * 32 * 4 +
           (S::REC_SMEM ? (size_t)W * rec_bufs<S, W>() * S::REC_F4 * 32 * 16 : 0);
}

template <class S, int W, int JS = 1>
cudaError_t launch_sym(int, const ForceArgs &a, cudaStream_t st) {
    constexpr int B = W * 32 * S::R;
    constexpr size_t smem = sym_smem<S, W, JS>();
    auto k = sym_kernel<S, W, JS, false>;
    auto kt = sym_kernel<S, W, JS, true>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(kt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int64_t nb = a.npad / B;
    if (nb * B != a.npad || nb != a.ntiles) return cudaErrorInvalidValue;
    if (a.tile_w > 0) {
        // one launch per tile, each a programmatic dependent of the one
        // before; then the last fold and the epilogue
        const int nt = sym_tile_count((int)nb, a.tile_w);
        if (nt != a.ntile) return cudaErrorInvalidValue;
        ForceArgs t = a;
        for (int s = 0; s < nt; ++s) {
            t.tile = s;
            const SymTile g = sym_tile(s, (int)nb, a.tile_w);
            cudaError_t e = launch_ex((const void *)kt, dim3((unsigned)g.items()), dim3(sym_threads<W, JS>()), smem,
                                      s == 0 ? a.pdl != 0 : true, t, st);
            if (e != cudaSuccess) return e;
        }
        return launch_ex((const void *)sym_tile_final_kernel<S, B>, dim3((unsigned)((a.n + 127) / 128)),
                         dim3(128), 0, true, t, st);
    }
    const unsigned items = (unsigned)(nb * (nb + 1) / 2);
    cudaError_t e = launch_ex((const void *)k, dim3(items), dim3(sym_threads<W, JS>()), smem, a.pdl != 0, a, st);
    if (e != cudaSuccess) return e;
    // the epilogue is a programmatic dependent of the pair kernel: its launch
    // overlaps the pair kernel's last wave, and it waits for its completion
    return launch_ex((const void *)sym_finish_kernel<S>, dim3((unsigned)((a.n + 31) / 32)),
                     dim3(32 * S::NACC), 0, true, a, st);
}

template <class S, int W, int JS = 1>
int occ_sym(int) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, sym_kernel<S, W, JS, false>, sym_threads<W, JS>(),
                                                      sym_smem<S, W, JS>()) !=
        cudaSuccess)
        return 0;
    return b;
}

// Shape (nt, r) = (threads per CTA, bodies per lane); the block is nt x r.
const ForceEntry kAccel[] = {
    {32, SymAccel::R, &launch_sym<SymAccel, 1>, &occ_sym<SymAccel, 1>},   // blocks of 256
    // blocks of 256, two warps splitting each block pair's j-chunks (64 threads x 4 bodies)
    {64, SymAccel::R / 2, &launch_sym<SymAccel, 1, 2>, &occ_sym<SymAccel, 1, 2>},
    {64, SymAccel::R, &launch_sym<SymAccel, 2>, &occ_sym<SymAccel, 2>},   // blocks of 512
    {128, SymAccel::R, &launch_sym<SymAccel, 4>, &occ_sym<SymAccel, 4>},  // blocks of 1024
};
const ForceEntry kComp[] = {
    {32, SymComp::R, &launch_sym<SymComp, 1>, &occ_sym<SymComp, 1>},   // blocks of 256
    {64, SymComp::R / 2, &launch_sym<SymComp, 1, 2>, &occ_sym<SymComp, 1, 2>},  // 256, j-chunks split
    {64, SymComp::R, &launch_sym<SymComp, 2>, &occ_sym<SymComp, 2>},   // blocks of 512
    {128, SymComp::R, &launch_sym<SymComp, 4>, &occ_sym<SymComp, 4>},  // blocks of 1024
};
const ForceEntry kVjpComp[] = {
    {64, SymVjpComp::R, &launch_sym<SymVjpComp, 2>, &occ_sym<SymVjpComp, 2>},   // blocks of 256
    {128, SymVjpComp::R, &launch_sym<SymVjpComp, 4>, &occ_sym<SymVjpComp, 4>},  // blocks of 512
};
const ForceEntry kVjp[] = {
    {64, SymVjp::R, &launch_sym<SymVjp, 2>, &occ_sym<SymVjp, 2>},   // blocks of 256
    {128, SymVjp::R, &launch_sym<SymVjp, 4>, &occ_sym<SymVjp, 4>},  // blocks of 512
};

}  // namespace

const ForceEntry *table_sym(int *count) {
    *count = (int)(sizeof(kAccel) / sizeof(kAccel[0]));
    return kAccel;
}

const ForceEntry *table_comp_sym(int *count) {
    *count = (int)(sizeof(kComp) / sizeof(kComp[0]));
    return kComp;
}

const ForceEntry *table_vjp_comp_sym(int *count) {
    *count = (int)(sizeof(kVjpComp) / sizeof(kVjpComp[0]));
    return kVjpComp;
}

const ForceEntry *table_vjp_sym(int *count) {
    *count = (int)(sizeof(kVjp) / sizeof(kVjp[0]));
    return kVjp;
}

}  // namespace nb
