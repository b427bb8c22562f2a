// Transforms of a few hundred to a few thousand points in shared memory, in
// the Stockham form: natural order in and out, two buffers used in turn, each
// pass giving every thread one sub-transform of radix 8, 6, 5, 4, 3 or 2 in
// registers (the in-plane grid transforms and the FP32 line transforms).
#pragma once

#include <cstdint>
#include <vector>

namespace fbc {

constexpr int kMaxPass = 8;

// One transform length and its passes: pass p has radix R[p], Ns[p] = the product of the earlier
// radices, NR[p] = N / R[p] work items per sequence, twiddle step N / (Ns R); divisions by NR and Ns
// as multiply-high, add and shift (m, l).
struct Fft1D {
    int N = 0, np = 0;
    int R[kMaxPass], Ns[kMaxPass], NR[kMaxPass], tstep[kMaxPass];
    unsigned mNR[kMaxPass], mNs[kMaxPass];
    int lNR[kMaxPass], lNs[kMaxPass];
};

namespace fft {

// n / d for 0 <= n < 2^31 with (m, l) from div_magic(d)
__device__ __forceinline__ int fdiv(int n, unsigned m, int l) {
    return (int)((__umulhi((unsigned)n, m) + (unsigned)n) >> l);
}

inline void div_magic(int d, unsigned* m, int* l) {
    int s = 0;
    while ((1LL << s) < d) s++;
    *l = s;
    *m = (unsigned)((((unsigned long long)1 << 32) * (((unsigned long long)1 << s) - (unsigned long long)d)) /
                    (unsigned long long)d + 1ULL);
}

// fewest passes of radix 8, 6, 5, 4, 3, 2 with product n (empty if n has another prime factor)
inline std::vector<int> radix_passes(int n) {
    static const int kRad[6] = {8, 6, 5, 4, 3, 2};
    std::vector<std::vector<int>> best(n + 1);
    std::vector<bool> ok(n + 1, false);
    ok[1] = true;
    for (int m = 2; m <= n; m++) {
        if (n % m) continue;
        for (int R : kRad)
            if (m % R == 0 && ok[m / R] && (!ok[m] || best[m / R].size() + 1 < best[m].size())) {
                best[m] = best[m / R];
                best[m].push_back(R);
                ok[m] = true;
            }
    }
    return ok[n] ? best[n] : std::vector<int>();
}

// The passes of a transform of exactly N points (np = 0 if N has a prime factor above 5).
inline Fft1D make_fft(int N) {
    Fft1D F;
    const std::vector<int> p = radix_passes(N);
    F.N = N;
    F.np = (int)p.size() <= kMaxPass ? (int)p.size() : 0;
    int Ns = 1;
    for (int q = 0; q < F.np; q++) {
        F.R[q] = p[q], F.Ns[q] = Ns, F.NR[q] = N / p[q], F.tstep[q] = N / (Ns * p[q]);
        div_magic(F.NR[q], &F.mNR[q], &F.lNR[q]);
        div_magic(Ns, &F.mNs[q], &F.lNs[q]);
        Ns *= p[q];
    }
    return F;
}

__device__ __forceinline__ float fmx(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmx(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename C> __device__ __forceinline__ C mkc(decltype(C::x) x, decltype(C::x) y) {
    C c;
    c.x = x, c.y = y;
    return c;
}

template <typename C> __device__ __forceinline__ C cmul(C a, C w) {
    return mkc<C>(fmx(a.x, w.x, -a.y * w.y), fmx(a.x, w.y, a.y * w.x));
}

// Shared-memory index with one pad slot after every 8 complex numbers: the early Stockham passes store
// with strides of 8 and 64 elements, which would otherwise hit the same banks.
__device__ __forceinline__ int sx(int i) { return i + (i >> 3); }
__host__ __device__ inline int padded(int n) { return n + (n >> 3) + 1; }

template <bool INV, typename C> __device__ __forceinline__ C add(C a, C b) { return mkc<C>(a.x + b.x, a.y + b.y); }
template <bool INV, typename C> __device__ __forceinline__ C sub(C a, C b) { return mkc<C>(a.x - b.x, a.y - b.y); }
// times -i (forward) or +i (inverse)
template <bool INV, typename C> __device__ __forceinline__ C rot(C a) {
    return INV ? mkc<C>(-a.y, a.x) : mkc<C>(a.y, -a.x);
}

template <bool INV, typename C> __device__ __forceinline__ void dft2(C* v) {
    const C t = v[0];
    v[0] = add<INV>(t, v[1]), v[1] = sub<INV>(t, v[1]);
}

template <bool INV, typename C> __device__ __forceinline__ void dft4(C& v0, C& v1, C& v2, C& v3) {
    const C a0 = add<INV>(v0, v2), a1 = sub<INV>(v0, v2), a2 = add<INV>(v1, v3), a3 = rot<INV>(sub<INV>(v1, v3));
    v0 = add<INV>(a0, a2), v1 = add<INV>(a1, a3), v2 = sub<INV>(a0, a2), v3 = sub<INV>(a1, a3);
}

// 8-point transform from two 4-point ones (even and odd inputs) and the factors exp(-+ i pi k / 4)
template <bool INV, typename C> __device__ __forceinline__ void dft8(C* v) {
    using R = decltype(C::x);
    const R h = (R)0.70710678118654752440;
    C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<INV>(e0, e1, e2, e3);
    dft4<INV>(o0, o1, o2, o3);
    o1 = INV ? mkc<C>((o1.x - o1.y) * h, (o1.x + o1.y) * h) : mkc<C>((o1.x + o1.y) * h, (o1.y - o1.x) * h);
    o2 = rot<INV>(o2);
    o3 = INV ? mkc<C>(-(o3.x + o3.y) * h, (o3.x - o3.y) * h) : mkc<C>((o3.y - o3.x) * h, -(o3.x + o3.y) * h);
    v[0] = add<INV>(e0, o0), v[4] = sub<INV>(e0, o0);
    v[1] = add<INV>(e1, o1), v[5] = sub<INV>(e1, o1);
    v[2] = add<INV>(e2, o2), v[6] = sub<INV>(e2, o2);
    v[3] = add<INV>(e3, o3), v[7] = sub<INV>(e3, o3);
}

template <bool INV, typename C> __device__ __forceinline__ void dft3(C& v0, C& v1, C& v2) {
    using R = decltype(C::x);
    const R h = (R)0.86602540378443864676;  // sin(2 pi / 3)
    const C t1 = add<INV>(v1, v2), d = sub<INV>(v1, v2);
    const C t2 = INV ? mkc<C>(-d.y * h, d.x * h) : mkc<C>(d.y * h, -d.x * h);  // -+ i h (v1 - v2)
    const C m = mkc<C>(v0.x - (R)0.5 * t1.x, v0.y - (R)0.5 * t1.y);
    v0 = add<INV>(v0, t1), v1 = add<INV>(m, t2), v2 = sub<INV>(m, t2);
}

template <bool INV, typename C> __device__ __forceinline__ void dft5(C* v) {
    using R = decltype(C::x);
    const R c1 = (R)0.30901699437494742410, c2 = (R)-0.80901699437494742410;  // cos(2 pi / 5), cos(4 pi / 5)
    const R s1 = (R)0.95105651629515357212, s2 = (R)0.58778525229247312917;   // sin(2 pi / 5), sin(4 pi / 5)
    const C t1 = add<INV>(v[1], v[4]), t2 = add<INV>(v[2], v[3]), t3 = sub<INV>(v[1], v[4]), t4 = sub<INV>(v[2], v[3]);
    const C a1 = mkc<C>(v[0].x + c1 * t1.x + c2 * t2.x, v[0].y + c1 * t1.y + c2 * t2.y);
    const C a2 = mkc<C>(v[0].x + c2 * t1.x + c1 * t2.x, v[0].y + c2 * t1.y + c1 * t2.y);
    const C b1 = mkc<C>(s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y);
    const C b2 = mkc<C>(s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y);
    // forward: y1 = a1 - i b1, y2 = a2 - i b2, y3 = a2 + i b2, y4 = a1 + i b1 (inverse: i -> -i)
    const C ib1 = rot<INV>(b1), ib2 = rot<INV>(b2);
    v[0] = mkc<C>(v[0].x + t1.x + t2.x, v[0].y + t1.y + t2.y);
    v[1] = add<INV>(a1, ib1), v[4] = sub<INV>(a1, ib1);
    v[2] = add<INV>(a2, ib2), v[3] = sub<INV>(a2, ib2);
}

// 6 points from two 3-point transforms (even and odd inputs) and the factors exp(-+ i pi k / 3)
template <bool INV, typename C> __device__ __forceinline__ void dft6(C* v) {
    using R = decltype(C::x);
    const R h = (R)0.86602540378443864676;
    C e0 = v[0], e1 = v[2], e2 = v[4], o0 = v[1], o1 = v[3], o2 = v[5];
    dft3<INV>(e0, e1, e2);
    dft3<INV>(o0, o1, o2);
    // w1 = 1/2 -+ i h, w2 = -1/2 -+ i h
    const R sg = INV ? (R)1 : (R)-1;
    o1 = mkc<C>((R)0.5 * o1.x - sg * h * o1.y, (R)0.5 * o1.y + sg * h * o1.x);
    o2 = mkc<C>((R)-0.5 * o2.x - sg * h * o2.y, (R)-0.5 * o2.y + sg * h * o2.x);
    v[0] = add<INV>(e0, o0), v[3] = sub<INV>(e0, o0);
    v[1] = add<INV>(e1, o1), v[4] = sub<INV>(e1, o1);
    v[2] = add<INV>(e2, o2), v[5] = sub<INV>(e2, o2);
}

// One Stockham pass (pass q of F, radix R) over nseq sequences of length N: work item j of a
// sequence reads x[j + r N/R], twiddles by exp(-+2 pi i r k / (Ns R)) with k = j mod Ns, transforms
// in registers and writes y[(j - k) R + k + r Ns].  tw[m] = exp(-2 pi i m / N), m < N.
template <int R, bool INV, typename C>
__device__ __forceinline__ void stockham_pass(const C* in, C* out, int nseq, const Fft1D& F, int q,
                                              const C* __restrict__ tw) {
    const int N = F.N, NR = F.NR[q], Ns = F.Ns[q], tstep = F.tstep[q];
    const unsigned mNR = F.mNR[q], mNs = F.mNs[q];
    const int lNR = F.lNR[q], lNs = F.lNs[q];
    for (int t = threadIdx.x; t < nseq * NR; t += blockDim.x) {
        const int seq = fdiv(t, mNR, lNR), j = t - seq * NR, k = j - fdiv(j, mNs, lNs) * Ns;
        const int x0 = seq * N + j;
        C v[R];
#pragma unroll
        for (int r = 0; r < R; r++) v[r] = in[sx(x0 + r * NR)];
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; r++) {
                C w = __ldg(tw + r * k * tstep);
                if (INV) w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        if (R == 8) dft8<INV>(v);
        else if (R == 6) dft6<INV>(v);
        else if (R == 5) dft5<INV>(v);
        else if (R == 4) dft4<INV>(v[0], v[1], v[2], v[3]);
        else if (R == 3) dft3<INV>(v[0], v[1], v[2]);
        else dft2<INV>(v);
        const int y0 = seq * N + (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; r++) out[sx(y0 + r * Ns)] = v[r];
    }
}

// nseq transforms of length F.N in a (natural order, padded index); b is scratch of the same size.
// Returns the buffer that holds the result.  Starts and ends at a barrier.
template <bool INV, typename C>
__device__ C* fft_smem(C* a, C* b, int nseq, const Fft1D& F, const C* __restrict__ tw) {
    for (int q = 0; q < F.np; q++) {
        switch (F.R[q]) {
            case 8: stockham_pass<8, INV>(a, b, nseq, F, q, tw); break;
            case 6: stockham_pass<6, INV>(a, b, nseq, F, q, tw); break;
            case 5: stockham_pass<5, INV>(a, b, nseq, F, q, tw); break;
            case 4: stockham_pass<4, INV>(a, b, nseq, F, q, tw); break;
            case 3: stockham_pass<3, INV>(a, b, nseq, F, q, tw); break;
            default: stockham_pass<2, INV>(a, b, nseq, F, q, tw); break;
        }
        __syncthreads();
        C* t = a;
        a = b, b = t;
    }
    return a;
}

}  // namespace fft
}  // namespace fbc
