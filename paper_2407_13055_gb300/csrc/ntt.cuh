// Radix-2 negacyclic NTT building blocks (Sec. 2.2, Sec. 4.2 "(I)NTT").
//
// A limb of N = H * W residues is viewed as H rows of W contiguous words,
// H = Ec^2 and W = Er^2. The forward transform (Cooley-Tukey, psi powers
// merged into the twiddles, natural order in, bit-reversed order out) runs its
// first log2 H stages down the columns ("column phase") and its last log2 W
// stages along the rows ("row phase"); the inverse (Gentleman-Sande) runs the
// row phase first. Each phase is two register passes of log2 E stages on E
// values per thread with one shared-memory transpose between them:
//   A layout: thread jj of a row (column) holds elements jj + E*i,
//   B layout: thread jj holds elements E*jj + i,  i = 0 .. E-1.
// The twiddle of stage s (m = 2^s butterfly blocks) and block b is
// tw[m + b] = psi^brev(m + b); inside a pass whose first stage has
// m0 = 2^(stages done before) and whose thread covers outer block o, local
// stage s uses index (m0 + o) 2^s + (i >> (log2 E - s)).
#pragma once
#include <cstdint>

#include "arith.cuh"

namespace ckks {

template <int E>
struct Log2 {
  static constexpr int v = (E <= 1) ? 0 : 1 + Log2<E / 2>::v;
};
template <>
struct Log2<1> {
  static constexpr int v = 0;
};

// Forward pass: log2 E Cooley-Tukey stages on E registers.
template <int E, bool LAZY>
__device__ __forceinline__ void ct_pass(uint32_t (&x)[E], const uint2* __restrict__ tw, uint32_t base,
                                        uint32_t q) {
  constexpr int e = Log2<E>::v;
#pragma unroll
  for (int s = 0; s < e; ++s) {
    const int half = E >> (s + 1);
#pragma unroll
    for (int b = 0; b < (1 << s); ++b) {
      const uint2 w = __ldg(&tw[(base << s) + b]);
#pragma unroll
      for (int r = 0; r < half; ++r) {
        const int i0 = b * 2 * half + r;
        ct_bfly<LAZY>(x[i0], x[i0 + half], w.x, w.y, q);
      }
    }
  }
}

// Inverse pass: the same stages in reverse order with Gentleman-Sande
// butterflies and the inverse twiddles psi^-brev(m + b).
template <int E, bool LAZY>
__device__ __forceinline__ void gs_pass(uint32_t (&x)[E], const uint2* __restrict__ itw, uint32_t base,
                                        uint32_t q) {
  constexpr int e = Log2<E>::v;
#pragma unroll
  for (int s = e - 1; s >= 0; --s) {
    const int half = E >> (s + 1);
#pragma unroll
    for (int b = 0; b < (1 << s); ++b) {
      const uint2 w = __ldg(&itw[(base << s) + b]);
#pragma unroll
      for (int r = 0; r < half; ++r) {
        const int i0 = b * 2 * half + r;
        gs_bfly<LAZY>(x[i0], x[i0 + half], w.x, w.y, q);
      }
    }
  }
}

// Row transpose through shared memory. buf holds one row with position
// l + l/E (conflict-free for both layouts). The E threads of a row sit in one
// warp, so a warp barrier suffices.
template <int E>
__device__ __forceinline__ void row_a_to_b(uint32_t (&x)[E], uint32_t* buf, int jj) {
#pragma unroll
  for (int i = 0; i < E; ++i) buf[jj + (E + 1) * i] = x[i];
  __syncwarp();
#pragma unroll
  for (int i = 0; i < E; ++i) x[i] = buf[(E + 1) * jj + i];
  __syncwarp();
}

template <int E>
__device__ __forceinline__ void row_b_to_a(uint32_t (&x)[E], uint32_t* buf, int jj) {
#pragma unroll
  for (int i = 0; i < E; ++i) buf[(E + 1) * jj + i] = x[i];
  __syncwarp();
#pragma unroll
  for (int i = 0; i < E; ++i) x[i] = buf[jj + (E + 1) * i];
  __syncwarp();
}

// Barrier over the threads that share a column tile: the whole block
// (bar == 0) or named barrier `bar` over `nthr` threads (a slice of the block).
__device__ __forceinline__ void tile_sync(int bar, int nthr) {
  if (bar == 0) __syncthreads();
  else asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(nthr) : "memory");
}

// Column transpose for a tile of TC columns: buf[(h + h/E) * TC + c].
// The E threads of a column are spread over several warps: tile barrier.
template <int E, int TC>
__device__ __forceinline__ void col_a_to_b(uint32_t (&x)[E], uint32_t* buf, int jj, int c, int bar = 0,
                                           int nthr = 0) {
#pragma unroll
  for (int i = 0; i < E; ++i) buf[(jj + (E + 1) * i) * TC + c] = x[i];
  tile_sync(bar, nthr);
#pragma unroll
  for (int i = 0; i < E; ++i) x[i] = buf[((E + 1) * jj + i) * TC + c];
  tile_sync(bar, nthr);
}

template <int E, int TC>
__device__ __forceinline__ void col_b_to_a(uint32_t (&x)[E], uint32_t* buf, int jj, int c, int bar = 0,
                                           int nthr = 0) {
#pragma unroll
  for (int i = 0; i < E; ++i) buf[((E + 1) * jj + i) * TC + c] = x[i];
  tile_sync(bar, nthr);
#pragma unroll
  for (int i = 0; i < E; ++i) x[i] = buf[(jj + (E + 1) * i) * TC + c];
  tile_sync(bar, nthr);
}

// Phases. H = EC^2 rows of W = ER^2 words.
// Row phase, forward: x in A layout of row h in, B layout out.
template <int ER, int H, bool LAZY>
__device__ __forceinline__ void row_fwd(uint32_t (&x)[ER], uint32_t* buf, const uint2* tw, int h, int jj,
                                        uint32_t q) {
  ct_pass<ER, LAZY>(x, tw, H + h, q);
  row_a_to_b<ER>(x, buf, jj);
  ct_pass<ER, LAZY>(x, tw, (uint32_t)(H + h) * ER + jj, q);
}

// Row phase, inverse: B layout in, A layout out.
template <int ER, int H, bool LAZY>
__device__ __forceinline__ void row_inv(uint32_t (&x)[ER], uint32_t* buf, const uint2* itw, int h, int jj,
                                        uint32_t q) {
  gs_pass<ER, LAZY>(x, itw, (uint32_t)(H + h) * ER + jj, q);
  row_b_to_a<ER>(x, buf, jj);
  gs_pass<ER, LAZY>(x, itw, H + h, q);
}

// Column phase, forward: A layout along h in, B layout out.
template <int EC, int TC, bool LAZY>
__device__ __forceinline__ void col_fwd(uint32_t (&x)[EC], uint32_t* buf, const uint2* tw, int jj, int c,
                                        uint32_t q, int bar = 0, int nthr = 0) {
  ct_pass<EC, LAZY>(x, tw, 1, q);
  col_a_to_b<EC, TC>(x, buf, jj, c, bar, nthr);
  ct_pass<EC, LAZY>(x, tw, EC + jj, q);
}

// Column phase, inverse: B layout in, A layout out.
template <int EC, int TC, bool LAZY>
__device__ __forceinline__ void col_inv(uint32_t (&x)[EC], uint32_t* buf, const uint2* itw, int jj, int c,
                                        uint32_t q, int bar = 0, int nthr = 0) {
  gs_pass<EC, LAZY>(x, itw, EC + jj, q);
  col_b_to_a<EC, TC>(x, buf, jj, c, bar, nthr);
  gs_pass<EC, LAZY>(x, itw, 1, q);
}

// Vector loads/stores of E consecutive words (B layout of a row).
template <int E>
__device__ __forceinline__ void load_vec(uint32_t (&x)[E], const uint32_t* __restrict__ p) {
  if constexpr (E % 4 == 0) {
    const uint4* v = reinterpret_cast<const uint4*>(p);
#pragma unroll
    for (int i = 0; i < E / 4; ++i) {
      uint4 t = __ldg(v + i);
      x[4 * i] = t.x; x[4 * i + 1] = t.y; x[4 * i + 2] = t.z; x[4 * i + 3] = t.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < E; ++i) x[i] = __ldg(p + i);
  }
}

// Streaming load (read once: cache-streaming, evict-first policy).
template <int E>
__device__ __forceinline__ void load_vec_stream(uint32_t (&x)[E], const uint32_t* __restrict__ p) {
  if constexpr (E % 4 == 0) {
    const uint4* v = reinterpret_cast<const uint4*>(p);
#pragma unroll
    for (int i = 0; i < E / 4; ++i) {
      const uint4 t = __ldcs(v + i);
      x[4 * i] = t.x; x[4 * i + 1] = t.y; x[4 * i + 2] = t.z; x[4 * i + 3] = t.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < E; ++i) x[i] = __ldg(p + i);
  }
}

template <int E>
__device__ __forceinline__ void store_vec(uint32_t* p, const uint32_t (&x)[E]) {
  if constexpr (E % 4 == 0) {
    uint4* v = reinterpret_cast<uint4*>(p);
#pragma unroll
    for (int i = 0; i < E / 4; ++i) v[i] = make_uint4(x[4 * i], x[4 * i + 1], x[4 * i + 2], x[4 * i + 3]);
  } else {
#pragma unroll
    for (int i = 0; i < E; ++i) p[i] = x[i];
  }
}

}  // namespace ckks
