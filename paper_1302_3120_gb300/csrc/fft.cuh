// fft.cuh — register/shared-memory Stockham FFT building blocks for sm_103a.
//
// A length-Q transform (Q = 2^q, 16 <= Q <= 8192) is computed by Q/R threads that
// each hold R complex64 values in registers (R = 32, or 16 when Q = 16).
// "Canonical order" means thread t holds v[s] = element t + s*(Q/R), s = 0..R-1;
// it is the input order of the first stage and the output order of the last
// stage, so a transform's first stage consumes values loaded straight from global
// memory and its last stage feeds a store (or the next transform) without a
// shared-memory round trip.  A length-8192 transform is 8 x 32 x 32: three
// register stages and two shared-memory exchanges.
//
// Stage (radix RS, span NS): butterfly b reads elements b + r*(Q/RS), multiplies
// them by W_{NS*RS}^{r*(b mod NS)}, does a length-RS DFT and writes element
// (b/NS)*NS*RS + (b mod NS) + r*NS (Stockham autosort).  Exchanges go through
// shared memory in place (all reads of a stage complete before its writes); the
// padding after each exchange (one spare slot per 2^shift elements) was chosen by
// simulating the bank pattern of every write/read of the exchange.
//
// Twiddles W_8192^m come from two small tables (W^m = hi[m >> 7] * lo[m & 127])
// computed in FP64 on the host and rounded once; inside a radix-32 butterfly the
// powers r = 1, 8, 16, 24 are looked up and the others formed by one or two
// products, so every twiddle is within a few ulp.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace csar {

constexpr int kTwN = 8192;      // twiddle table length (largest transform)
constexpr int kTwLo = 128;
constexpr int kTwHi = kTwN / kTwLo;

__host__ __device__ constexpr int regs_for(int q) { return q >= 32 ? 32 : 16; }
// values per thread in the column passes (more warps per SM to hide shared-memory latency)
__host__ __device__ constexpr int col_regs(int q) { return 16; }

// Complex add and subtract as one packed two-lane FP32 instruction each (sm_100-class
// f32x2 arithmetic; every lane rounds to nearest like the scalar instruction, so the
// results are the same).  -DCSAR_SCALAR_COMPLEX restores the scalar pairs.
#ifdef CSAR_SCALAR_COMPLEX
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
#else
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
  float2 o;
  asm("{\n\t.reg .b64 pa, pb, pd;\n\t"
      "mov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
      "add.rn.f32x2 pd, pa, pb;\n\tmov.b64 {%0, %1}, pd;\n\t}"
      : "=f"(o.x), "=f"(o.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return o;
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
  float2 o;
  asm("{\n\t.reg .b64 pa, pb, pd;\n\t"
      "mov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
      "sub.rn.f32x2 pd, pa, pb;\n\tmov.b64 {%0, %1}, pd;\n\t}"
      : "=f"(o.x), "=f"(o.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return o;
}
#endif
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float cabs2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }

// multiply by W_4^1: -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 mul_w4(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// cos(2 pi j / 32), j in [0, 32)
__device__ __forceinline__ constexpr float cos32(int j) {
  j &= 31;
  if (j > 16) j = 32 - j;
  float sgn = 1.f;
  if (j > 8) { j = 16 - j; sgn = -1.f; }
  float c = j == 0 ? 1.0f
          : j == 1 ? 0.98078528040323044913f
          : j == 2 ? 0.92387953251128675613f
          : j == 3 ? 0.83146961230254523708f
          : j == 4 ? 0.70710678118654752440f
          : j == 5 ? 0.55557023301960222474f
          : j == 6 ? 0.38268343236508977173f
          : j == 7 ? 0.19509032201612826785f
                   : 0.0f;
  return sgn * c;
}

// a * W_RS^k  (W = exp(-2 pi i / RS) forward, conjugate for the inverse), k constant
template <int RS, bool INV>
__device__ __forceinline__ float2 twiddle_const(float2 a, int k) {
  const int j = (k * (32 / RS)) & 31;   // angle 2 pi j / 32
  if (j == 0) return a;
  if (j == 8) return mul_w4<INV>(a);
  if (j == 16) return make_float2(-a.x, -a.y);
  if (j == 24) return mul_w4<!INV>(a);
  const float c = cos32(j);
  const float s = INV ? cos32(j - 8) : -cos32(j - 8);  // sin(2 pi j/32) = cos(2 pi (j-8)/32)
  if (j == 4 || j == 12 || j == 20 || j == 28) {         // (+-1 +- i)/sqrt(2): 2 mul + 2 add
    const float p = a.x * c, q = a.y * c;                 // |c| = |s|
    return (c == s) ? make_float2(p - q, p + q) : make_float2(p + q, q - p);
  }
  return make_float2(fmaf(a.x, c, -a.y * s), fmaf(a.x, s, a.y * c));
}

// Radix-2 butterfly with a constant twiddle: lo = e + o W, hi = e - o W, W = W_RS^k
// (conjugate for the inverse).  Trivial twiddles (1, -i, -1, +i) keep the plain product;
// for the others W = c + i s is split as m (r + i) or m (1 + i r) with m the larger of
// |c|, |s| and |r| <= 1 (the tangent form of the butterfly): u = o (W / m) takes two
// FMAs and lo, hi = e +- m u four more, 6 FP32 operations per butterfly instead of 8.
template <int RS, bool INV>
__device__ __forceinline__ void bfly_const(float2 e, float2 o, int k, float2& lo, float2& hi) {
  const int j = (k * (32 / RS)) & 31;   // angle 2 pi j / 32
  if (j % 8 == 0) {
    const float2 t = twiddle_const<RS, INV>(o, k);
    lo = cadd(e, t);
    hi = csub(e, t);
    return;
  }
  const float c = cos32(j);
  const float s = INV ? cos32(j - 8) : -cos32(j - 8);   // sin(2 pi j/32) = cos(2 pi (j-8)/32)
  float2 u;
  float m;
  if (fabsf(c) >= fabsf(s)) {   // W = c (1 + i r), r = s / c
    const float r = s / c;
    u = make_float2(fmaf(-o.y, r, o.x), fmaf(o.x, r, o.y));
    m = c;
  } else {                      // W = s (r + i), r = c / s
    const float r = c / s;
    u = make_float2(fmaf(o.x, r, -o.y), fmaf(o.y, r, o.x));
    m = s;
  }
  lo = make_float2(fmaf(m, u.x, e.x), fmaf(m, u.y, e.y));
  hi = make_float2(fmaf(-m, u.x, e.x), fmaf(-m, u.y, e.y));
}

// In-place length-RS DFT on a[0..RS-1], natural order in and out (radix-2 DIT).
template <int RS, bool INV>
struct Dft {
  static __device__ __forceinline__ void run(float2* a) {
    float2 e[RS / 2], o[RS / 2];
#pragma unroll
    for (int i = 0; i < RS / 2; ++i) { e[i] = a[2 * i]; o[i] = a[2 * i + 1]; }
    Dft<RS / 2, INV>::run(e);
    Dft<RS / 2, INV>::run(o);
#pragma unroll
    for (int k = 0; k < RS / 2; ++k) {
      bfly_const<RS, INV>(e[k], o[k], k, a[k], a[k + RS / 2]);
    }
  }
};
template <bool INV>
struct Dft<4, INV> {
  static __device__ __forceinline__ void run(float2* a) {
    const float2 t0 = cadd(a[0], a[2]), t1 = csub(a[0], a[2]);
    const float2 t2 = cadd(a[1], a[3]), t3 = mul_w4<INV>(csub(a[1], a[3]));
    a[0] = cadd(t0, t2);
    a[2] = csub(t0, t2);
    a[1] = cadd(t1, t3);
    a[3] = csub(t1, t3);
  }
};
template <bool INV>
struct Dft<2, INV> {
  static __device__ __forceinline__ void run(float2* a) {
    const float2 t = a[0];
    a[0] = cadd(t, a[1]);
    a[1] = csub(t, a[1]);
  }
};

// W_8192^m (forward) or its conjugate (inverse) from the two-level table in smem.
template <bool INV>
__device__ __forceinline__ float2 twiddle_tab(const float2* tw, int m) {
  m &= (kTwN - 1);
  float2 w = cmul(tw[kTwLo + (m >> 7)], tw[m & (kTwLo - 1)]);
  if (INV) w.y = -w.y;
  return w;
}

// Copy the 192-entry twiddle table to shared memory (call before the first stage).
__device__ __forceinline__ void load_twiddles(float2* tw_sm, const float2* __restrict__ tw_g) {
  for (int i = threadIdx.x; i < kTwLo + kTwHi; i += blockDim.x) tw_sm[i] = tw_g[i];
}

// Radix of the first stage: Q = first * R^k.
__host__ __device__ constexpr int first_radix(int q, int r) {
  int f = q;
  while (f > r) f /= r;
  return f == 1 ? r : f;
}

// Element (w, n) of W transforms of length Q.
//   Row layout: transform w is contiguous (w*Q + n).
//   Col layout: element n of all W transforms is contiguous (n*W + w).
// SHIFT: one padding slot every 2^SHIFT elements.
template <int Q, int W, bool COL>
struct Layout {
  static constexpr int kW = W;
  static constexpr int kStride = COL ? W : 1;   // flat distance between n and n+1
  static __device__ __forceinline__ int flat(int w, int n) { return COL ? n * W + w : w * Q + n; }
  template <int SHIFT>
  static __device__ __forceinline__ int at(int w, int n) {
    const int f = flat(w, n);
    return f + (f >> SHIFT);
  }
  static constexpr int kSmemElems = (Q * W) + (Q * W) / 16;
};

// Padded addresses of the RS elements n0 + r*DN (r = 0..RS-1) of transform w.  When the
// flat step is a multiple of 2^SHIFT the padding is a compile-time offset from one
// base address, which keeps the address arithmetic out of the register file.
template <class L, int SHIFT, int DN>
struct Strided {
  static constexpr int kFlat = DN * L::kStride;
  static constexpr bool kAffine = (kFlat % (1 << SHIFT)) == 0;
  static constexpr int kStep = kFlat + (kFlat >> SHIFT);
  static __device__ __forceinline__ int base(int w, int n0) { return L::template at<SHIFT>(w, n0); }
  static __device__ __forceinline__ int at(int w, int n0, int base_addr, int r) {
    if constexpr (kAffine) return base_addr + r * kStep;
    else return L::template at<SHIFT>(w, n0 + r * DN);
  }
};

// Padding of the exchange written by a stage of radix RS.
template <bool COL, int RS>
struct PadShift {
  static constexpr int value = (!COL && RS == 32) ? 5 : 4;
};

constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v / 2); }

// First exchange of a column layout (written by the first stage, radix RS0, read by
// the second, radix RS1).  The first stage writes elements RS0*b + r, which puts the
// W columns of 16/W consecutive butterflies b on the same banks; instead of padding,
// the r-field of the flat index f = n*W + w is XORed with the low bits of b:
//     slot(f) = f ^ (W * ((f >> log2(W*RS0)) & M)),   M = min(16/W, RS0) - 1,
// a permutation inside each group of RS0 rows.  Both the write (per-thread base, M+1
// address registers, compile-time offsets) and the second-stage read (per-thread
// base, affine in r) stay free of per-element address arithmetic.
template <int Q, int W, int RS0, int RS1>
struct Swz {
  static constexpr int M = ((16 / W) < RS0 ? (16 / W) : RS0) - 1;
  static constexpr int kShift = ilog2(W * RS0);
  static constexpr bool kOn = M > 0 && RS0 > 1 && (Q / (RS0 * RS1)) % (M + 1) == 0;
  static __device__ __forceinline__ int slot(int f) { return kOn ? (f ^ (W * ((f >> kShift) & M))) : f; }
};
constexpr int kSwzPad = -1;   // PS / OPS value marking the swizzled first exchange

template <int RS, bool INV>
__device__ __forceinline__ void apply_twiddles(float2* a, const float2* tw, int step) {
  // a[r] *= W^(r*step) (W = W_8192), r = 1..RS-1
  float2 w1 = twiddle_tab<INV>(tw, step);
  if constexpr (RS <= 8) {
    float2 w = w1;
#pragma unroll
    for (int r = 1; r < RS; ++r) {
      a[r] = cmul(a[r], w);
      if (r + 1 < RS) w = cmul(w, w1);
    }
  } else {
    float2 p[8];
    p[1] = w1;
#pragma unroll
    for (int r = 2; r < 8; ++r) p[r] = cmul(p[r - 1], w1);
#pragma unroll
    for (int r = 1; r < 8; ++r) a[r] = cmul(a[r], p[r]);
#pragma unroll
    for (int blk = 8; blk < RS; blk += 8) {
      const float2 anc = twiddle_tab<INV>(tw, blk * step);
      a[blk] = cmul(a[blk], anc);
#pragma unroll
      for (int r = 1; r < 8; ++r) a[blk + r] = cmul(a[blk + r], cmul(anc, p[r]));
    }
  }
}

// All stages of one length-Q transform, starting from span NS.  v is in canonical
// order on entry when NS == 1 and on exit.  sm: the transform group's shared
// buffer (laid out by L); tw: shared twiddle table.  PS: padding of the exchange
// this stage reads (ignored when NS == 1).
template <int Q, int R, bool INV, class L, bool COL, int NS, int PS>
struct Stages {
  static __device__ __forceinline__ void run(float2 (&v)[R], float2* sm, const float2* tw,
                                             int t, int w) {
    constexpr int RS = (NS == 1) ? first_radix(Q, R) : R;
    constexpr int G = R / RS;             // butterflies per thread
    constexpr int QR = Q / R;             // threads per transform
    if constexpr (NS > 1 && PS == kSwzPad) {
      // second stage of a column transform: read the swizzled first exchange
      using S = Swz<Q, L::kW, NS, RS>;
      __syncthreads();
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const int b = t + g * QR;
        const int ba = S::slot(L::flat(w, b));   // the XOR term does not depend on r
#pragma unroll
        for (int r = 0; r < RS; ++r) v[g + r * G] = sm[ba + r * (Q / RS) * L::kStride];
      }
    } else if constexpr (NS > 1) {
      __syncthreads();
      using RD = Strided<L, PS, Q / RS>;
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const int b = t + g * QR;
        const int ba = RD::base(w, b);
#pragma unroll
        for (int r = 0; r < RS; ++r) v[g + r * G] = sm[RD::at(w, b, ba, r)];
      }
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int b = t + g * QR;
      float2 a[RS];
#pragma unroll
      for (int r = 0; r < RS; ++r) a[r] = v[g + r * G];
      if constexpr (NS > 1) {
        const int k = b & (NS - 1);
        apply_twiddles<RS, INV>(a, tw, k * (kTwN / (NS * RS)));
      }
      Dft<RS, INV>::run(a);
#pragma unroll
      for (int r = 0; r < RS; ++r) v[g + r * G] = a[r];
    }
    if constexpr (NS * RS < Q) {
      using S = Swz<Q, L::kW, RS, (NS * RS < Q) ? R : 1>;
      constexpr bool kSwz = COL && NS == 1 && S::kOn;
      constexpr int OPS = kSwz ? kSwzPad : PadShift<COL, RS>::value;
      __syncthreads();
      if constexpr (kSwz) {
        // element RS*b + r goes to slot (RS*b + (r ^ (b & M)))*W + w
        constexpr int M = S::M;
#pragma unroll
        for (int g = 0; g < G; ++g) {
          const int b = t + g * QR;
          const int base = L::flat(w, RS * b);
          int ad[M + 1];
#pragma unroll
          for (int j = 0; j <= M; ++j) ad[j] = base + L::kW * (j ^ (b & M));
#pragma unroll
          for (int r = 0; r < RS; ++r) sm[ad[r & M] + L::kW * (r & ~M)] = v[g + r * G];
        }
      } else {
        using WR = Strided<L, OPS, NS>;
#pragma unroll
        for (int g = 0; g < G; ++g) {
          const int b = t + g * QR;
          const int k = b & (NS - 1);
          const int n0 = (b / NS) * NS * RS + k;
          const int ba = WR::base(w, n0);
#pragma unroll
          for (int r = 0; r < RS; ++r) sm[WR::at(w, n0, ba, r)] = v[g + r * G];
        }
      }
      Stages<Q, R, INV, L, COL, NS * RS, OPS>::run(v, sm, tw, t, w);
    }
  }
};

// Full transform, canonical order in and out.  Contains __syncthreads() when Q > R:
// every thread of the block must call it.
template <int Q, bool INV, class L, bool COL, int R = regs_for(Q)>
__device__ __forceinline__ void fft(float2 (&v)[R], float2* sm, const float2* tw, int t, int w) {
  Stages<Q, R, INV, L, COL, 1, 4>::run(v, sm, tw, t, w);
}

}  // namespace csar
