// linefft.cuh -- the register line FFT of the 2D line kernels and of the
// cluster engine: a line of F = 2^LF points held by F/8 threads, 8 points
// each (Eq. fftp36 / Eq. fftp35 transforms along one axis, the line symbol of
// Eq. energy-discrete-FP between the forward and the inverse transform).
//
// Thread j holds the points j + s F/8 (s = 0..7).  The transform is a
// Stockham autosort FFT of radix-8 stages and, when LF is not a multiple of
// 3, one radix-4 or radix-2 tail stage; every stage reads the points
// j + s F/8, so the natural order of the input, of the spectrum (symbol
// multiply) and of the output is the register order, and shared memory is
// touched only by the exchanges between stages (two alternating buffers, one
// barrier of the line's threads per exchange).
#pragma once
#include "ops_impl.cuh"

namespace gpe {

template <typename T, int LF>
struct LineFFT {
  using C = typename C2t<T>::type;
  static constexpr int F = 1 << LF;
  static constexpr int TPL = F / 8;                 // threads per line
  static constexpr int N8 = LF / 3;                 // radix-8 stages
  static constexpr int TAIL = LF % 3;               // 1: radix-2 tail stage, 2: radix-4 tail stage
  // line pitch of the exchange buffers (complex): room for F points, and
  // = 8 (mod 16) so that neighbouring lines start half a bank row apart
  static constexpr int P = ((F + F / 16 + 15) & ~15) + 8;
  // twiddles e^{-2 pi i n / F} come from the table tws (shared memory); in
  // float32 the thread's 13-17 twiddles are also kept in registers
  static constexpr bool TW_REG = sizeof(T) == 4;
  C w8[TW_REG && N8 > 1 ? N8 - 1 : 1][7];
  C wt[TW_REG ? 6 : 1];
  const C* tws;
  int j;

  // twiddle r of radix-8 stage st (>= 1): e^{-2 pi i r k / (8 Ns)}, k = j mod Ns
  __device__ __forceinline__ C tw8(int st, int r) const {
    if constexpr (TW_REG) return w8[st - 1][r - 1];
    const int Ns = 1 << (3 * st);
    return tws[(r * (j & (Ns - 1))) << (LF - 3 - 3 * st)];
  }
  // tail twiddles: radix-4 (i = r - 1 for butterfly j, r + 2 for j + F/8),
  // radix-2 (i = u)
  __device__ __forceinline__ C twt(int i) const {
    if constexpr (TW_REG) return wt[i];
    if constexpr (TAIL == 2) return tws[i < 3 ? (i + 1) * j : (i - 2) * (j + TPL)];
    return tws[j + i * TPL];
  }

  __device__ __forceinline__ void init(int jj, const C* table) {
    j = jj;
    tws = table;
    if constexpr (TW_REG) {
#pragma unroll
      for (int st = 1; st < N8; ++st) {
        const int Ns = 1 << (3 * st);
        const int k = j & (Ns - 1);
#pragma unroll
        for (int r = 1; r < 8; ++r) w8[st - 1][r - 1] = table[(r * k) << (LF - 3 - 3 * st)];
      }
      if constexpr (TAIL == 2) {
#pragma unroll
        for (int r = 1; r < 4; ++r) {
          wt[r - 1] = table[r * j];
          wt[r + 2] = table[r * (j + TPL)];
        }
      } else if constexpr (TAIL == 1) {
#pragma unroll
        for (int u = 0; u < 4; ++u) wt[u] = table[j + u * TPL];
      }
    }
  }

  // Forward DFT (unnormalised) of this thread's line: v[s] = x[j + s F/8] in,
  // X[j + s F/8] out.  ex(par, m) is the shared-memory slot of point m of this
  // line in exchange buffer par; par alternates between the two buffers.
  template <typename Ex>
  __device__ __forceinline__ void forward(C (&v)[8], const Ex& ex, int& par) const {
#pragma unroll
    for (int st = 0; st < N8; ++st) {
      if (st > 0) {
#pragma unroll
        for (int r = 1; r < 8; ++r) v[r] = cmul(v[r], tw8(st, r));
      }
      dft8<C, false>(v);
      if (st + 1 < N8 || TAIL) {
        const int Ns = 1 << (3 * st);
        const int k = j & (Ns - 1);
        const int mb = ((j - k) << 3) + k;
#pragma unroll
        for (int r = 0; r < 8; ++r) *ex(par, mb + r * Ns) = v[r];
        ex.sync();
#pragma unroll
        for (int s = 0; s < 8; ++s) v[s] = *ex(par, j + s * TPL);
        par ^= 1;
      }
    }
    if constexpr (TAIL == 2) {
      // butterflies j (slots 0,2,4,6) and j + F/8 (slots 1,3,5,7)
      v[2] = cmul(v[2], twt(0));
      v[4] = cmul(v[4], twt(1));
      v[6] = cmul(v[6], twt(2));
      v[3] = cmul(v[3], twt(3));
      v[5] = cmul(v[5], twt(4));
      v[7] = cmul(v[7], twt(5));
      dft4<C, false>(v[0], v[2], v[4], v[6]);
      dft4<C, false>(v[1], v[3], v[5], v[7]);
    } else if constexpr (TAIL == 1) {
      // butterflies j + u F/8 (slots u, u + 4)
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        v[u + 4] = cmul(v[u + 4], twt(u));
        dft2<C, false>(v[u], v[u + 4]);
      }
    }
  }

  // T applied to the line: forward DFT, symbol(m) and conjugation, forward DFT,
  // conjugation (= inverse DFT of the symbol times the spectrum).
  template <typename Ex, typename Sym>
  __device__ __forceinline__ void apply(C (&v)[8], const Ex& ex, int& par, Sym sym) const {
    forward(v, ex, par);
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const T sy = sym(j + s * TPL);
      v[s].x = sy * v[s].x;
      v[s].y = -sy * v[s].y;
    }
    forward(v, ex, par);
#pragma unroll
    for (int s = 0; s < 8; ++s) v[s].y = -v[s].y;
  }
};

// Slot of point m in a line's exchange row: bits 3-6 of m XORed into bits 0-3,
// a bijection within each 128-point block.  A radix-8 stage with sub-length
// Ns stores thread j's eight points at 8(j - j mod Ns) + j mod Ns + r Ns, and
// the next stage loads the points j + s F/8; with this swizzle every such warp
// access touches the minimum number of shared-memory wavefronts for 8- and
// 16-byte complex values (checked by enumerating the banks of every warp
// access for F = 64 ... 1024), where padding one slot per 16 points leaves the
// stores of the Ns = 8 stage two-way conflicted.
__device__ __forceinline__ int lidx(int m) { return m ^ ((m >> 3) & 15); }

// Exchange slots of a line stored contiguously (row pitch P, swizzled index):
// the x-kernel, where the threads of a warp share a line.  Only the line's own
// threads touch its rows, so an exchange waits for them alone: a named
// barrier over the line's warps, or the warp itself when a line fits in one.
template <typename C, int P>
struct ExRow {
  C* base;          // line row in buffer 0
  int pstride;      // buffer 1 - buffer 0
  int bar_id;       // named barrier of the line (1 + line in the CTA)
  int bar_n;        // threads of the line
  __device__ __forceinline__ C* operator()(int par, int m) const { return base + par * pstride + lidx(m); }
  __device__ __forceinline__ void sync() const {
    if (bar_n <= 32) __syncwarp();
    else asm volatile("bar.sync %0, %1;\n" ::"r"(bar_id), "r"(bar_n) : "memory");
  }
};

// The line symbol: c2 lam^2 + c1 coord lam, lam = dlam * (m or m - F).
template <typename T, int F>
struct LineSym {
  T c2, c1c, dl;
  __device__ __forceinline__ T operator()(int m) const {
    const T lm = dl * (T)(m < (F >> 1) ? m : m - F);
    return (c2 * lm + c1c) * lm;
  }
};

}  // namespace gpe
