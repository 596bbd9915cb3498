// Line FFTs held entirely in one thread's registers, for lengths known at compile
// time.  The self-sorting Stockham stages of fft.cu are unrolled completely, so
// every array index and twiddle index is a constant: no shared memory, no
// barriers, no index arithmetic at run time.  Used for the strided x and y axes,
// where neighbouring threads own neighbouring lines and every load and store of
// a warp is coalesced without staging.
#pragma once

#include <cmath>

#include "common.cuh"

namespace tdlz {

// Twiddles of one line length, passed BY VALUE as a kernel parameter: every index
// into it is a compile-time constant after unrolling, so each twiddle is read
// straight from the kernel-parameter constant bank as an instruction operand
// (no loads, no per-device constant-memory set-up).  w[t] = exp(+2 pi i t / N).
template <class T, int N> struct RegTw {
  cx<T> w[N];
};

// Host-side table, computed once per (type, length) in double precision.
template <class T, int N> inline const RegTw<T, N> &regtw() {
  static const RegTw<T, N> tab = [] {
    RegTw<T, N> t;
    const double two_pi = 6.283185307179586476925286766559;
    for (int i = 0; i < N; ++i) {
      t.w[i].x = (T)std::cos(two_pi * i / N);
      t.w[i].y = (T)std::sin(two_pi * i / N);
    }
    return t;
  }();
  return tab;
}

// twiddle exp(+2 pi i t / N); DIR < 0 conjugates
template <class T, int DIR, int N>
__device__ __forceinline__ cx<T> rtw(const RegTw<T, N> &tw, int t) {
  cx<T> w = tw.w[t];
  if (DIR < 0) w.y = -w.y;
  return w;
}

template <class T, int R, int DIR, int N>
__device__ __forceinline__ void rdft(cx<T> (&v)[R], const RegTw<T, N> &tw) {
  if constexpr (R == 2) {
    cx<T> a = v[0];
    v[0] = cadd<T>(a, v[1]);
    v[1] = csub<T>(a, v[1]);
  } else if constexpr (R == 4) {
    cx<T> a = cadd<T>(v[0], v[2]), b = csub<T>(v[0], v[2]);
    cx<T> c = cadd<T>(v[1], v[3]), d = csub<T>(v[1], v[3]);
    cx<T> e = DIR > 0 ? mk<T>(-d.y, d.x) : mk<T>(d.y, -d.x);
    v[0] = cadd<T>(a, c);
    v[2] = csub<T>(a, c);
    v[1] = cadd<T>(b, e);
    v[3] = csub<T>(b, e);
  } else if constexpr (R == 3) {
    const cx<T> w3 = rtw<T, DIR, N>(tw, N / 3);
    cx<T> s = cadd<T>(v[1], v[2]), d = csub<T>(v[1], v[2]);
    cx<T> m = mk<T>(v[0].x + w3.x * s.x, v[0].y + w3.x * s.y);
    cx<T> r = mk<T>(-w3.y * d.y, w3.y * d.x);
    v[0] = cadd<T>(v[0], s);
    v[1] = cadd<T>(m, r);
    v[2] = csub<T>(m, r);
  } else {
    static_assert(R == 5, "radix");
    const cx<T> w5a = rtw<T, DIR, N>(tw, N / 5), w5b = rtw<T, DIR, N>(tw, (2 * N) / 5);
    cx<T> a1 = cadd<T>(v[1], v[4]), b1 = csub<T>(v[1], v[4]);
    cx<T> a2 = cadd<T>(v[2], v[3]), b2 = csub<T>(v[2], v[3]);
    T c1 = w5a.x, s1 = w5a.y, c2 = w5b.x, s2 = w5b.y;
    cx<T> m1 = mk<T>(v[0].x + c1 * a1.x + c2 * a2.x, v[0].y + c1 * a1.y + c2 * a2.y);
    cx<T> m2 = mk<T>(v[0].x + c2 * a1.x + c1 * a2.x, v[0].y + c2 * a1.y + c1 * a2.y);
    cx<T> p1 = mk<T>(-(s1 * b1.y + s2 * b2.y), s1 * b1.x + s2 * b2.x);
    cx<T> p2 = mk<T>(-(s2 * b1.y - s1 * b2.y), s2 * b1.x - s1 * b2.x);
    v[0] = cadd<T>(v[0], cadd<T>(a1, a2));
    v[1] = cadd<T>(m1, p1);
    v[4] = csub<T>(m1, p1);
    v[2] = cadd<T>(m2, p2);
    v[3] = csub<T>(m2, p2);
  }
}

// One Stockham stage a -> b: radix R, sub-transform length NS.
template <class T, int N, int R, int NS, int DIR>
__device__ __forceinline__ void rstage(const cx<T> (&a)[N], cx<T> (&b)[N],
                                       const RegTw<T, N> &tw) {
  constexpr int NR = N / R;
  constexpr int TS = N / (NS * R);
#pragma unroll
  for (int j = 0; j < NR; ++j) {
    const int k = j % NS;
    cx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = a[j + r * NR];
    if (k != 0) {
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmul<T>(v[r], rtw<T, DIR, N>(tw, (r * k * TS) % N));
    }
    rdft<T, R, DIR, N>(v, tw);
    const int ob = (j / NS) * NS * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) b[ob + r * NS] = v[r];
  }
}

template <class T, int N, int DIR, int NS, int R, int... Rs>
__device__ __forceinline__ void rstages(cx<T> (&a)[N], const RegTw<T, N> &tw) {
  cx<T> b[N];
  rstage<T, N, R, NS, DIR>(a, b, tw);
#pragma unroll
  for (int i = 0; i < N; ++i) a[i] = b[i];
  if constexpr (sizeof...(Rs) > 0) rstages<T, N, DIR, NS * R, Rs...>(a, tw);
}

// Radix plans of the lengths handled in registers (3, 4, 6, 8, 9, 15, 18 are the
// per-lane parts of lines split over two or three lanes).
template <int N> struct RegPlan;
template <> struct RegPlan<3> {
  template <class T, int DIR>
  __device__ static void run(cx<T> (&a)[3], const RegTw<T, 3> &tw) {
    rstages<T, 3, DIR, 1, 3>(a, tw);
  }
};
template <> struct RegPlan<4> {
  template <class T, int DIR>
  __device__ static void run(cx<T> (&a)[4], const RegTw<T, 4> &tw) {
    rstages<T, 4, DIR, 1, 4>(a, tw);
  }
};
template <> struct RegPlan<6> {
  template <class T, int DIR>
  __device__ static void run(cx<T> (&a)[6], const RegTw<T, 6> &tw) {
    rstages<T, 6, DIR, 1, 2, 3>(a, tw);
  }
};
template <> struct RegPlan<8> {
  template <class T, int DIR>
  __device__ static void run(cx<T> (&a)[8], const RegTw<T, 8> &tw) {
    rstages<T, 8, DIR, 1, 4, 2>(a, tw);
  }
};
template <> struct RegPlan<9> {
  template <class T, int DIR>
  __device__ static void run(cx<T> (&a)[9], const RegTw<T, 9> &tw) {
    rstages<T, 9, DIR, 1, 3, 3>(a, tw);
  }
};
template <> struct RegPlan<15> {
  template <class T, int DIR>
  __device__ static void run(cx<T> (&a)[15], const RegTw<T, 15> &tw) {
    rstages<T, 15, DIR, 1, 3, 5>(a, tw);
  }
};
template <> struct RegPlan<18> {
  template <class T, int DIR>
  __device__ static void run(cx<T> (&a)[18], const RegTw<T, 18> &tw) {
    rstages<T, 18, DIR, 1, 2, 3, 3>(a, tw);
  }
};
template <> struct RegPlan<12> {
  template <class T, int DIR>
  __device__ static void run(cx<T> (&a)[12], const RegTw<T, 12> &tw) {
    rstages<T, 12, DIR, 1, 4, 3>(a, tw);
  }
};
template <> struct RegPlan<16> {
  template <class T, int DIR>
  __device__ static void run(cx<T> (&a)[16], const RegTw<T, 16> &tw) {
    rstages<T, 16, DIR, 1, 4, 4>(a, tw);
  }
};
template <> struct RegPlan<24> {
  template <class T, int DIR>
  __device__ static void run(cx<T> (&a)[24], const RegTw<T, 24> &tw) {
    rstages<T, 24, DIR, 1, 4, 2, 3>(a, tw);
  }
};
template <> struct RegPlan<36> {
  template <class T, int DIR>
  __device__ static void run(cx<T> (&a)[36], const RegTw<T, 36> &tw) {
    rstages<T, 36, DIR, 1, 4, 3, 3>(a, tw);
  }
};
template <> struct RegPlan<45> {
  template <class T, int DIR>
  __device__ static void run(cx<T> (&a)[45], const RegTw<T, 45> &tw) {
    rstages<T, 45, DIR, 1, 3, 3, 5>(a, tw);
  }
};
template <> struct RegPlan<48> {
  template <class T, int DIR>
  __device__ static void run(cx<T> (&a)[48], const RegTw<T, 48> &tw) {
    rstages<T, 48, DIR, 1, 4, 4, 3>(a, tw);
  }
};

inline bool reg_fft_length(int n) {
  return n == 12 || n == 16 || n == 24 || n == 36 || n == 45 || n == 48;
}

}  // namespace tdlz
