// exdot.cuh -- exact, correctly rounded FP64 dot products on sm_103a using
// integer arithmetic only.
//
// Section 2 of arXiv 2404.13216 replaces residual replacement in p-BiCGStab by
// ExBLAS dot products: a long fixed-point accumulator fed by floating-point
// expansions, rounded once, independent of data partitioning and reduction
// order.  GB300 issues FP64 at roughly 2 FMA per clock per SM against about 64
// integer operations, so this engine keeps the long-accumulator idea but builds
// every stage from integer instructions:
//
//   1. decode both doubles into (sign, 53-bit integer mantissa, exponent) with
//      bit operations;
//   2. form the exact 106-bit mantissa product with four 32x32->64 multiplies;
//   3. add it, as a signed 256-bit two's-complement number, into a per-lane
//      register window whose bit position (the anchor) is shared by the warp;
//      a term above the window re-anchors it (after flushing), and terms below
//      it are deposited together into a temporary window anchored at their own
//      maximum, which is flushed at once;
//   4. at the end of a pass the warp sums its windows (butterfly with carries)
//      and adds the total into the CTA accumulator: 32-bit digits held in
//      int64 (carry-save), bit 0 of digit 0 weighing 2^-2148;
//   5. each CTA adds its touched digits into one global accumulator per dot
//      with 64-bit atomics (integer addition is associative, so arrival order
//      does not matter);
//   6. the last CTA to finish normalises the carries and rounds the exact sum
//      to the nearest double (ties to even, subnormals exact, overflow to inf).
//
// Every stage is exact, so the rounded value is RN(sum a_i b_i) whatever the
// grid shape, row assignment or batch composition.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pbcg {

constexpr int NDIG = 136;        // 32-bit digits; 136*32 = 4352 bits cover 2^-2148 .. 2^2048 plus carries
constexpr int WIN_WORDS = 8;     // per-lane window: 256-bit two's complement
constexpr int WIN_SMAX = 120;    // largest left shift of a 106-bit product inside the window (3 words + 24 bits)
constexpr int WIN_ROOM = 32;     // bits of room left above the warp maximum when anchoring
constexpr int WIN_UNSET = -(1 << 24);   // anchor of an empty window: every term is above it

// ---------------------------------------------------------------------------
// decode and exact product
// ---------------------------------------------------------------------------
struct Prod {
    uint32_t w0, w1, w2, w3;     // |a*b| mantissa product (< 2^106)
    uint32_t neg;                // 1 if a*b < 0
};

// ---------------------------------------------------------------------------
// CTA accumulator (shared memory) for ND dots
// ---------------------------------------------------------------------------
template <int ND>
struct CtaAcc {
    unsigned long long dig[ND][NDIG];   // carry-save signed digits (two's complement int64)
    int kmin[ND], kmax[ND];
    int nf[ND];
};

template <int ND>
__device__ __forceinline__ void cta_acc_init(CtaAcc<ND> &c)
{
    unsigned long long *d = &c.dig[0][0];
    for (int i = threadIdx.x; i < ND * NDIG; i += blockDim.x)
        d[i] = 0ull;
    if (threadIdx.x < ND) {
        c.kmin[threadIdx.x] = NDIG;
        c.kmax[threadIdx.x] = -1;
        c.nf[threadIdx.x] = 0;
    }
}

template <int ND>
__device__ __forceinline__ void cta_touch(CtaAcc<ND> &c, int d, int k0, int k1)
{
    atomicMin(&c.kmin[d], k0);
    atomicMax(&c.kmax[d], k1);
}

// ---------------------------------------------------------------------------
// per-lane window: 256-bit two's complement, LSB at bit `anchor` (warp-uniform)
//
// Headroom: a product shifted by at most WIN_SMAX bits is below 2^226; a lane
// adds fewer than 2^16 of them between flushes (one per tile of its CTA) and
// a warp sums 32 lanes, so totals stay below 2^247 and the sign bit (255) is
// never reached.
// ---------------------------------------------------------------------------
struct Win {
    uint32_t a[WIN_WORDS];
    int anchor;      // WIN_UNSET while unset
};

__device__ __forceinline__ void win_init(Win &w)
{
#pragma unroll
    for (int t = 0; t < WIN_WORDS; t++)
        w.a[t] = 0u;
    w.anchor = WIN_UNSET;
}

__device__ __forceinline__ void add256(uint32_t (&a)[WIN_WORDS], const uint32_t (&x)[WIN_WORDS])
{
    asm("add.cc.u32 %0, %0, %8;\n\t"
        "addc.cc.u32 %1, %1, %9;\n\t"
        "addc.cc.u32 %2, %2, %10;\n\t"
        "addc.cc.u32 %3, %3, %11;\n\t"
        "addc.cc.u32 %4, %4, %12;\n\t"
        "addc.cc.u32 %5, %5, %13;\n\t"
        "addc.cc.u32 %6, %6, %14;\n\t"
        "addc.u32 %7, %7, %15;"
        : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5]), "+r"(a[6]), "+r"(a[7])
        : "r"(x[0]), "r"(x[1]), "r"(x[2]), "r"(x[3]), "r"(x[4]), "r"(x[5]), "r"(x[6]), "r"(x[7]));
}

// Sum the windows of the warp (all lanes call) and add the total, anchored at
// bit `anchor`, into the CTA digits; leaves the window zero.
template <int ND>
__device__ __forceinline__ void win_flush_words(uint32_t (&a)[WIN_WORDS], int anchor, CtaAcc<ND> &c, int d)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        uint32_t y[WIN_WORDS];
#pragma unroll
        for (int t = 0; t < WIN_WORDS; t++)
            y[t] = __shfl_xor_sync(0xffffffffu, a[t], o);
        add256(a, y);
    }
    const int k = anchor >> 5;
    const uint32_t r = (uint32_t)(anchor & 31);
    const uint32_t sg = (uint32_t)((int)a[WIN_WORDS - 1] >> 31);
    const int lane = threadIdx.x & 31;
    // lane t (t <= WIN_WORDS) takes word t of (total << r)
    uint32_t lo = 0u, hi = 0u;
#pragma unroll
    for (int t = 0; t < WIN_WORDS; t++) {
        if (lane == t)
            hi = a[t];
        if (lane == t + 1)
            lo = a[t];
    }
    if (lane == WIN_WORDS)
        hi = sg;
    const uint32_t mine = (lane == 0) ? (hi << r) : __funnelshift_l(lo, hi, r);
    if (lane <= WIN_WORDS) {
        const unsigned long long v = (lane < WIN_WORDS) ? (unsigned long long)mine
                                                        : (unsigned long long)(long long)(int)mine;
        if (v != 0ull)
            atomicAdd(&c.dig[d][k + lane], v);
    }
    if (lane == 0)
        cta_touch(c, d, k, k + WIN_WORDS);
#pragma unroll
    for (int t = 0; t < WIN_WORDS; t++)
        a[t] = 0u;
}

template <int ND>
__device__ __forceinline__ void win_flush_reset(Win &w, CtaAcc<ND> &c, int d)
{
    win_flush_words<ND>(w.a, w.anchor, c, d);
}

// Sum the warp's windows and add the total into the CTA digits.  All lanes call.
template <int ND>
__device__ __forceinline__ void win_flush(Win &w, CtaAcc<ND> &c, int d)
{
    if (w.anchor < 0)
        return;                                           // warp-uniform: nothing deposited
    win_flush_words<ND>(w.a, w.anchor, c, d);
}

// ---------------------------------------------------------------------------
// operand-level interface: decode each double once, deposit products of
// decoded operands (a value shared by several dots is decoded only once)
// ---------------------------------------------------------------------------
constexpr int E_ZERO = -100000;    // exponent sentinel of a zero operand: its products drop out

struct Dec {
    uint32_t lo, hi;     // 53-bit integer mantissa: hi holds the top 21 bits (implicit bit included)
    int e;               // max(biased exponent, 1), or E_ZERO for +-0
    uint32_t s;          // sign bit
    bool nf;             // Inf or NaN
};

__device__ __forceinline__ Dec decode(double a)
{
    unsigned long long b = (unsigned long long)__double_as_longlong(a);
    uint32_t h = (uint32_t)(b >> 32);
    Dec d;
    d.lo = (uint32_t)b;
    uint32_t ef = (h >> 20) & 0x7ffu;
    d.nf = ef == 0x7ffu;
    d.hi = (h & 0xfffffu) | (ef ? 0x100000u : 0u);
    d.s = h >> 31;
    d.e = ((d.hi | d.lo) == 0u) ? E_ZERO : (ef ? (int)ef : 1);
    return d;
}

// exact product of two decoded operands (|a*b| words and sign; its LSB lies
// a.e + b.e - 2 bits above 2^-2148)
template <bool SQUARE>
__device__ __forceinline__ Prod dec_product(const Dec &a, const Dec &b)
{
    Prod p;
    unsigned long long p0 = (unsigned long long)a.lo * b.lo;
    unsigned long long m;
    if (SQUARE) {      // a == b: the two cross terms are equal (each < 2^53)
        m = (((unsigned long long)a.hi * b.lo) << 1) + (p0 >> 32);
    } else {
        m = (unsigned long long)a.hi * b.lo + (p0 >> 32);
        m = (unsigned long long)a.lo * b.hi + m;
    }
    unsigned long long h = (unsigned long long)a.hi * b.hi + (m >> 32);
    p.w0 = (uint32_t)p0;
    p.w1 = (uint32_t)m;
    p.w2 = (uint32_t)h;
    p.w3 = (uint32_t)(h >> 32);
    p.neg = SQUARE ? 0u : (a.s ^ b.s);
    return p;
}

// acc += (-1)^neg |p| 2^sh for 0 <= sh <= WIN_SMAX.  A negative term is added
// as its 256-bit one's complement plus one: the words of |p| << sh and the
// words around them are XORed with the sign mask, and the +1 enters as the
// carry into word 0, so no separate negation chain is needed.
template <bool SQUARE>
__device__ __forceinline__ void place_product(uint32_t (&acc)[WIN_WORDS], const Prod &p, int sh)
{
    const uint32_t r = (uint32_t)sh & 31u, q = (uint32_t)sh >> 5;
    const uint32_t m = SQUARE ? 0u : 0u - p.neg;
    const uint32_t u0 = (p.w0 << r) ^ m, u1 = __funnelshift_l(p.w0, p.w1, r) ^ m;
    const uint32_t u2 = __funnelshift_l(p.w1, p.w2, r) ^ m, u3 = __funnelshift_l(p.w2, p.w3, r) ^ m;
    const uint32_t u4 = __funnelshift_l(p.w3, 0u, r) ^ m;
    const bool q1 = q & 1u, q2 = q & 2u;
    // word t of the term: u[t-q] for t-q in 0..4, the mask elsewhere
    const uint32_t v0 = q1 ? m : u0, v1 = q1 ? u0 : u1, v2 = q1 ? u1 : u2;
    const uint32_t v3 = q1 ? u2 : u3, v4 = q1 ? u3 : u4, v5 = q1 ? u4 : m;
    uint32_t x[WIN_WORDS];
    x[0] = q2 ? m : v0;
    x[1] = q2 ? m : v1;
    x[2] = q2 ? v0 : v2;
    x[3] = q2 ? v1 : v3;
    x[4] = q2 ? v2 : v4;
    x[5] = q2 ? v3 : v5;
    x[6] = q2 ? v4 : m;
    x[7] = q2 ? v5 : m;
    if (SQUARE) {
        add256(acc, x);
    } else {
        uint32_t cf;
        asm("add.cc.u32 %8, %16, 0xffffffff;\n\t"      // carry = neg
            "addc.cc.u32 %0, %0, %9;\n\t"
            "addc.cc.u32 %1, %1, %10;\n\t"
            "addc.cc.u32 %2, %2, %11;\n\t"
            "addc.cc.u32 %3, %3, %12;\n\t"
            "addc.cc.u32 %4, %4, %13;\n\t"
            "addc.cc.u32 %5, %5, %14;\n\t"
            "addc.cc.u32 %6, %6, %15;\n\t"
            "addc.u32 %7, %7, %17;"
            : "+r"(acc[0]), "+r"(acc[1]), "+r"(acc[2]), "+r"(acc[3]), "+r"(acc[4]), "+r"(acc[5]), "+r"(acc[6]),
              "+r"(acc[7]), "=r"(cf)
            : "r"(x[0]), "r"(x[1]), "r"(x[2]), "r"(x[3]), "r"(x[4]), "r"(x[5]), "r"(x[6]), "r"(p.neg), "r"(x[7]));
    }
}

// Products below the warp's window: deposit them together into a temporary
// window anchored at the largest of them and flush it at once; repeat while
// some are still lower than that window.  All lanes call.
template <int ND, bool SQUARE>
__device__ __noinline__ void win_low(CtaAcc<ND> &c, int d, Prod p, int rem)
{
    while (__any_sync(0xffffffffu, rem >= 0)) {
        const int m = __reduce_max_sync(0xffffffffu, rem);
        const int anc = max(m - WIN_SMAX, 0);
        uint32_t t[WIN_WORDS];
#pragma unroll
        for (int q = 0; q < WIN_WORDS; q++)
            t[q] = 0u;
        const bool go = rem >= 0 && rem >= anc;
        if (go) {
            place_product<SQUARE>(t, p, rem - anc);
            rem = -1;
        }
        win_flush_words<ND>(t, anc, c, d);
    }
}

// A term a*b prepared for a window: its exact product, LSB offset (negative
// for zero operands and inactive lanes) and shift above the window's anchor;
// `odd` when it does not land inside the window (also while it is unset).
struct WinTerm {
    Prod p;
    int off, sh;
    bool odd;
};

template <bool SQUARE>
__device__ __forceinline__ WinTerm win_term(const Win &w, const Dec &a, const Dec &b, bool act, bool &nf)
{
    WinTerm t;
    nf |= act && (a.nf || b.nf);
    t.off = act ? a.e + b.e - 2 : -1;
    t.p = dec_product<SQUARE>(a, b);
    t.sh = t.off - w.anchor;
    t.odd = t.off >= 0 && (uint32_t)t.sh > (uint32_t)WIN_SMAX;
    return t;
}

// The common case, known warp-wide: every lane's term lands inside the window.
template <bool SQUARE>
__device__ __forceinline__ void win_put(Win &w, const WinTerm &t)
{
    if (t.off >= 0)
        place_product<SQUARE>(w.a, t.p, t.sh);
}

// Deposit a prepared term.  All 32 lanes of the warp call together.  The
// anchor is kept warp-uniform: a vote finds lanes whose term would not fit
// the top of the window; only then is the window flushed and re-anchored at
// the warp maximum.  Terms below the window take win_low.
template <int ND, bool SQUARE>
__device__ __forceinline__ void win_settle(Win &w, CtaAcc<ND> &c, int d, WinTerm t)
{
    if (!__any_sync(0xffffffffu, t.odd)) {
        win_put<SQUARE>(w, t);
        return;
    }
    const bool high = t.off >= 0 && t.sh > WIN_SMAX;
    if (__any_sync(0xffffffffu, high)) {             // re-anchor at the warp maximum
        const int m = __reduce_max_sync(0xffffffffu, t.off);
        if (w.anchor >= 0)
            win_flush_reset<ND>(w, c, d);
        w.anchor = max(m - WIN_SMAX + WIN_ROOM, 0);
        t.sh = t.off - w.anchor;                     // <= WIN_SMAX for every lane with off >= 0
    }
    const bool low = t.off >= 0 && t.sh < 0;
    if (t.off >= 0 && t.sh >= 0)
        place_product<SQUARE>(w.a, t.p, t.sh);
    if (__any_sync(0xffffffffu, low))
        win_low<ND, SQUARE>(c, d, t.p, low ? t.off : -1);
}

// Deposit a*b for decoded operands.  All 32 lanes of the warp call together.
template <int ND, bool SQUARE>
__device__ __forceinline__ void win_add(Win &w, CtaAcc<ND> &c, int d, const Dec &a, const Dec &b, bool act,
                                        bool &nf)
{
    win_settle<ND, SQUARE>(w, c, d, win_term<SQUARE>(w, a, b, act, nf));
}

// Deposit a*b.  Must be called by all 32 lanes of the warp together (the
// anchor is chosen with a warp reduction); `active` masks lanes with no term.
template <int ND>
__device__ __forceinline__ void win_deposit(Win &w, CtaAcc<ND> &c, int d, double a, double b, bool active,
                                            bool &nf)
{
    win_add<ND, false>(w, c, d, decode(a), decode(b), active, nf);
}

// ---------------------------------------------------------------------------
// global accumulator: one per dot, merged by integer atomics
// ---------------------------------------------------------------------------
struct GAcc {
    unsigned long long dig[NDIG];
    int kmin, kmax, nf, pad;
};

template <int ND>
__device__ __forceinline__ void cta_to_global(CtaAcc<ND> &c, GAcc *g)
{
    for (int d = 0; d < ND; d++) {
        int k0 = c.kmin[d], k1 = c.kmax[d];
        for (int k = k0 + (int)threadIdx.x; k <= k1; k += blockDim.x) {
            unsigned long long v = c.dig[d][k];
            if (v != 0ull)
                atomicAdd(&g[d].dig[k], v);
        }
        if (threadIdx.x == 0) {
            if (k1 >= k0) {
                atomicMin(&g[d].kmin, k0);
                atomicMax(&g[d].kmax, k1);
            }
            if (c.nf[d])
                atomicOr(&g[d].nf, 1);
        }
    }
}

// Round the exact sum held in digits dig[k0..k1] (signed carry-save 32-bit
// digits, bit 0 of digit 0 weighing 2^-2148; digits outside the range are 0)
// to the nearest double.  One thread; `scratch` is NDIG words.
__device__ __forceinline__ uint32_t bit_at(const uint32_t *w, int lo, int hi, int i)
{
    int k = i >> 5;
    if (k < lo || k > hi)
        return 0u;
    return (w[k] >> (i & 31)) & 1u;
}

static __device__ double round_digits(const unsigned long long *dig, int k0, int k1, int nf, uint32_t *scratch)
{
    if (nf)
        return __longlong_as_double(0x7ff8000000000000ll);
    if (k1 < k0)
        return 0.0;
    // carry normalisation from k0 upward; digits above k1 start at 0
    long long carry = 0;
    int top = k0;
    for (int k = k0; k < NDIG; k++) {
        long long v = (k <= k1) ? (long long)dig[k] : 0ll;
        // v + carry without overflow: |digit| < 2^62 and |carry| < 2^31 here
        long long s = v + carry;
        scratch[k] = (uint32_t)s;
        carry = s >> 32;
        top = k;
        // stop once the rest is pure sign extension of a canonical top word
        if (k >= k1 && ((carry == 0 && !(scratch[k] >> 31)) || (carry == -1 && (scratch[k] >> 31))))
            break;
    }
    bool negv = carry < 0;
    if (negv) {
        // magnitude = -value over digits k0..top (infinite sign extension above)
        uint32_t c1 = 1u;
        for (int k = k0; k <= top; k++) {
            uint32_t x = ~scratch[k];
            unsigned long long s = (unsigned long long)x + c1;
            scratch[k] = (uint32_t)s;
            c1 = (uint32_t)(s >> 32);
        }
    }
    int hk = -1;
    for (int k = top; k >= k0; k--) {
        if (scratch[k] != 0u) {
            hk = k;
            break;
        }
    }
    if (hk < 0)
        return 0.0;
    int h = hk * 32 + 31 - __clz(scratch[hk]);
    int lsb = max(h - 52, 1074);
    // m = bits lsb..h (at most 53): the three words from lsb's word up hold
    // them, and every bit above h is 0
    auto word = [&](int k) -> unsigned long long { return (k >= k0 && k <= top) ? scratch[k] : 0u; };
    const int kl = lsb >> 5, sl = lsb & 31;
    const unsigned long long lo64 = word(kl) | (word(kl + 1) << 32);
    unsigned long long m = sl ? (lo64 >> sl) | (word(kl + 2) << (64 - sl)) : lo64;
    uint32_t rb = bit_at(scratch, k0, top, lsb - 1);
    uint32_t st = 0u;
    int sk = (lsb - 1) >> 5;
    for (int k = k0; k < sk && k <= top; k++)
        st |= scratch[k];
    if (sk >= k0 && sk <= top)
        st |= scratch[sk] & ((1u << ((lsb - 1) & 31)) - 1u);
    if (rb && (st || (m & 1ull)))
        m += 1ull;
    // value = m * 2^(lsb - 2148); biased exponent field = lsb - 1074 (+1 via the implicit bit)
    long long ef = (long long)(lsb - 1074);
    unsigned long long bits = ((unsigned long long)ef << 52) + m;
    if (bits >= 0x7ff0000000000000ull)
        bits = 0x7ff0000000000000ull;            // overflow rounds to infinity
    if (negv)
        bits |= 0x8000000000000000ull;
    return __longlong_as_double((long long)bits);
}

// The same rounding as round_digits, by all 32 lanes of one warp (returns the
// value in every lane).  Carry normalisation runs on 32 digits at a time:
// each lane holds one digit; the part of it above bit 31 moves one lane up
// (shuffles), after which every remaining carry is -1, 0 or +1, and those are
// settled at once by a carry-lookahead over the warp (ballots) -- no carry
// ripples lane by lane; the top lane's part carries into the next 32 digits.
// The lowest and highest nonzero words and the sticky bits below the
// rounding position come from ballots.  Every step is exact, so the result is
// round_digits' bit for bit.
static __device__ double round_digits_warp(const unsigned long long *dig, int k0, int k1, int nf, uint32_t *scratch)
{
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    if (nf)
        return __longlong_as_double(0x7ff8000000000000ll);
    if (k1 < k0)
        return 0.0;
    // 1. scratch[k0 .. top] := the two's complement words of the sum; stop once
    //    the words above are pure sign extension (carry 0 over a clear top bit,
    //    or -1 over a set one)
    long long cin = 0;
    int top = k0;
    for (int kc = k0; kc < NDIG; kc += 32) {
        const int k = kc + lane;
        long long d = (k <= k1) ? (long long)dig[k] : 0ll;
        if (lane == 0)
            d += cin;
        // move each digit's part above bit 31 one lane up (the top lane's out
        // of the chunk): |digit| < 2^62, so what a lane then holds lies in
        // (-2^30, 2^32 + 2^30) and its own carry is -1, 0 or +1
        const long long hi = d >> 32;
        const long long below = __shfl_up_sync(FULL, hi, 1);    // (every lane shuffles; lane 0 ignores it)
        long long out = __shfl_sync(FULL, hi, 31);
        d = (long long)(uint32_t)d + (lane == 0 ? 0ll : below);
        const int c1 = (int)(d >> 32);                       // -1, 0 or 1, into the next lane
        out += __shfl_sync(FULL, c1, 31);
        const int c1_below = __shfl_up_sync(FULL, c1, 1);
        const int inc = lane == 0 ? 0 : c1_below;
        uint32_t w = (uint32_t)d;
        // add the +1 carries, then the -1 borrows, each with a lookahead over
        // the warp: lane i is bit i; g generates (overflows by itself), p
        // propagates (overflows with one more); the carries into the lanes are
        // the carries of the integer addition g + (g | p)
        {
            const unsigned g = __ballot_sync(FULL, inc == 1 && w == 0xffffffffu);
            w += inc == 1 ? 1u : 0u;
            const unsigned p = __ballot_sync(FULL, w == 0xffffffffu);
            const unsigned long long sum = (unsigned long long)g + (unsigned long long)(g | p);
            const unsigned into = (unsigned)sum ^ (p & ~g);
            w += (into >> lane) & 1u;
            out += (long long)(sum >> 32);
        }
        {
            const unsigned g = __ballot_sync(FULL, inc == -1 && w == 0u);
            w -= inc == -1 ? 1u : 0u;
            const unsigned p = __ballot_sync(FULL, w == 0u);
            const unsigned long long sum = (unsigned long long)g + (unsigned long long)(g | p);
            const unsigned into = (unsigned)sum ^ (p & ~g);
            w -= (into >> lane) & 1u;
            out -= (long long)(sum >> 32);
        }
        if (k < NDIG)
            scratch[k] = w;
        cin = out;
        top = min(kc + 31, NDIG - 1);
        const uint32_t tw = __shfl_sync(FULL, w, 31);
        if (kc + 31 >= k1 && ((cin == 0 && !(tw >> 31)) || (cin == -1 && (tw >> 31))))
            break;
    }
    __syncwarp();
    const bool negv = cin < 0;
    if (negv) {
        // magnitude: words below the lowest nonzero one stay 0, that one is
        // negated, every word above it is inverted
        bool seen = false;
        for (int c = k0; c <= top; c += 32) {
            const int k = c + lane;
            const uint32_t w = (k <= top) ? scratch[k] : 0u;
            const unsigned nz = __ballot_sync(FULL, k <= top && w != 0u);
            uint32_t r;
            if (seen) {
                r = ~w;
            } else {
                const int low = nz ? __ffs(nz) - 1 : 32;
                r = lane < low ? 0u : (lane == low ? 0u - w : ~w);
            }
            seen = seen || nz != 0u;
            if (k <= top)
                scratch[k] = r;
        }
        __syncwarp();
    }
    // 2. the highest nonzero word
    int hk = -1;
    for (int c = top; c >= k0 && hk < 0; c -= 32) {
        const int k = c - lane;
        const unsigned nz = __ballot_sync(FULL, k >= k0 && scratch[k] != 0u);
        if (nz)
            hk = c - (__ffs(nz) - 1);
    }
    if (hk < 0)
        return 0.0;
    const int h = hk * 32 + 31 - __clz(scratch[hk]);
    const int lsb = max(h - 52, 1074);
    auto word = [&](int k) -> unsigned long long { return (k >= k0 && k <= top) ? scratch[k] : 0u; };
    const int kl = lsb >> 5, sl = lsb & 31;
    const unsigned long long lo64 = word(kl) | (word(kl + 1) << 32);
    unsigned long long m = sl ? (lo64 >> sl) | (word(kl + 2) << (64 - sl)) : lo64;
    const uint32_t rb = bit_at(scratch, k0, top, lsb - 1);
    // sticky: any bit below lsb - 1
    const int sk = (lsb - 1) >> 5;
    bool st = false;
    for (int c = k0; c < sk && c <= top; c += 32) {
        const int k = c + lane;
        st = st || __any_sync(FULL, k < sk && k <= top && scratch[k] != 0u);
    }
    if (sk >= k0 && sk <= top)
        st = st || (scratch[sk] & ((1u << ((lsb - 1) & 31)) - 1u)) != 0u;
    if (rb && (st || (m & 1ull)))
        m += 1ull;
    long long ef = (long long)(lsb - 1074);
    unsigned long long bits = ((unsigned long long)ef << 52) + m;
    if (bits >= 0x7ff0000000000000ull)
        bits = 0x7ff0000000000000ull;
    if (negv)
        bits |= 0x8000000000000000ull;
    return __longlong_as_double((long long)bits);
}

// Round the ND global accumulators g[0..ND-1] and reset them; every thread of
// the CTA calls.  All ND * NDIG digits (the untouched ones are 0) and the
// non-finite flags are loaded in one round trip to L2 -- every thread issues
// its loads before any store -- into the CTA accumulator c (free at this
// point: its contents were merged into g); the range each dot's rounding
// scans is that of its nonzero digits.  Warp d rounds dot d, the ND warps
// side by side.  dv[d] receives the rounded dots.
template <int ND>
__device__ void gacc_round_reset_cta(GAcc *g, CtaAcc<ND> &c, uint32_t (*scratch)[NDIG], double *dv)
{
    __syncthreads();
    if (threadIdx.x < ND) {
        c.kmin[threadIdx.x] = NDIG;
        c.kmax[threadIdx.x] = -1;
    }
    int nf = 0;
    if (threadIdx.x < ND)
        nf = *((volatile int *)&g[threadIdx.x].nf);
    // position i of the flattened (dot, digit) range: dot i / NDIG, digit i % NDIG
    constexpr int PER = (ND * NDIG + 255) / 256;
    unsigned long long v[PER];
#pragma unroll
    for (int j = 0; j < PER; j++) {
        const int i = (int)threadIdx.x + j * (int)blockDim.x;
        const int d = i / NDIG, k = i - d * NDIG;
        v[j] = i < ND * NDIG ? __ldcg(&g[d].dig[k]) : 0ull;
    }
    __syncthreads();                                 // (c.kmin / c.kmax initialised)
    if (threadIdx.x < ND)
        c.nf[threadIdx.x] = nf;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < PER; j++) {
        const int i = (int)threadIdx.x + j * (int)blockDim.x;
        const int d = i / NDIG, k = i - d * NDIG;
        const bool nz = i < ND * NDIG && v[j] != 0ull;
        if (i < ND * NDIG) {
            c.dig[d][k] = v[j];
            if (nz)
                g[d].dig[k] = 0ull;                  // every nonzero digit cleared, NaN results included
        }
        // the warp's lowest and highest nonzero digit of each dot it covers: its
        // lanes hold consecutive positions, so at most two dots (those of dot d0
        // form a prefix, the next dot starts at digit 0); one shared atomic per
        // bound instead of one per digit
        const unsigned mall = __ballot_sync(0xffffffffu, nz);
        const unsigned pre = __ballot_sync(0xffffffffu, d == __shfl_sync(0xffffffffu, d, 0));
        const int d0 = __shfl_sync(0xffffffffu, d, 0), kl0 = __shfl_sync(0xffffffffu, k, 0);
        const unsigned m0 = mall & pre, m1 = mall & ~pre;
        if (lane == 0) {
            if (m0) {
                atomicMin(&c.kmin[d0], kl0 + (__ffs(m0) - 1));
                atomicMax(&c.kmax[d0], kl0 + (31 - __clz(m0)));
            }
            if (m1) {
                const int L = __popc(pre);           // the lane holding digit 0 of dot d0 + 1
                atomicMin(&c.kmin[d0 + 1], (__ffs(m1) - 1) - L);
                atomicMax(&c.kmax[d0 + 1], (31 - __clz(m1)) - L);
            }
        }
    }
    for (int i = (int)threadIdx.x + PER * (int)blockDim.x; i < ND * NDIG; i += blockDim.x) {
        const int d = i / NDIG, k = i - d * NDIG;    // (a CTA of fewer than 256 threads)
        const unsigned long long w = __ldcg(&g[d].dig[k]);
        c.dig[d][k] = w;
        if (w != 0ull) {
            g[d].dig[k] = 0ull;
            atomicMin(&c.kmin[d], k);
            atomicMax(&c.kmax[d], k);
        }
    }
    __syncthreads();
    if ((int)(threadIdx.x >> 5) < ND) {
        const int d = threadIdx.x >> 5;
        const double r = round_digits_warp(c.dig[d], c.kmin[d], c.kmax[d], c.nf[d], scratch[d]);
        if ((threadIdx.x & 31) == 0) {
            dv[d] = r;
            g[d].kmin = NDIG;
            g[d].kmax = -1;
            g[d].nf = 0;
        }
    }
    __syncthreads();
}

}  // namespace pbcg
