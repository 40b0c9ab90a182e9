// Warp-level reductions shared by the factor and apply kernels.
#pragma once

namespace tsqr {

__host__ __device__ constexpr int pow2ceil(int x) { return x <= 1 ? 1 : 2 * pow2ceil((x + 1) / 2); }

// Transpose-reduce over the 16 lanes of a half-warp: each lane holds C partial sums
// (C a power of two <= 16). Stage s exchanges half of the values with the lane whose
// bit (8 >> s) differs and adds, until one value is left, then plain butterflies
// finish the sum. The lane ends with the half-warp total of value `idx`.
template <int C, typename R>
__device__ __forceinline__ R treduce16(R (&v)[C], int hl, int &idx) {
  idx = 0;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int m = 8 >> s;
    const int cs = (C >> s) > 1 ? (C >> s) : 1;
    if (cs > 1) {
      const int half = cs >> 1;
      const bool up = (hl & m) != 0;
#pragma unroll
      for (int i = 0; i < C / 2; ++i) {
        if (i < half) {
          const R send = up ? v[i] : v[i + half];
          const R keep = up ? v[i + half] : v[i];
          v[i] = keep + __shfl_xor_sync(0xffffffffu, send, m);
        }
      }
      if (up) idx += half;
    } else {
      v[0] += __shfl_xor_sync(0xffffffffu, v[0], m);
    }
  }
  return v[0];
}

// Transpose-reduce over a full warp: each lane holds C partial sums (C a power of two
// <= 32). Stage s exchanges half of the remaining values with the lane whose bit
// (16 >> s) differs and adds, until one value is left; plain butterflies then finish the
// sum. Each lane ends with the warp total of value idx.
template <int C, typename R>
__device__ __forceinline__ R treduce32(R (&v)[C], int lane, int &idx) {
  idx = 0;
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const int m = 16 >> s;
    const int cs = (C >> s) > 1 ? (C >> s) : 1;
    if (cs > 1) {
      const int half = cs >> 1;
      const bool up = (lane & m) != 0;
#pragma unroll
      for (int i = 0; i < C / 2; ++i) {
        if (i < half) {
          const R send = up ? v[i] : v[i + half];
          const R keep = up ? v[i + half] : v[i];
          v[i] = keep + __shfl_xor_sync(0xffffffffu, send, m);
        }
      }
      if (up) idx += half;
    } else {
      v[0] += __shfl_xor_sync(0xffffffffu, v[0], m);
    }
  }
  return v[0];
}

// Lowest lane that holds the total of value c after treduce32<C>; the total is
// replicated on the 32 / C lanes above it.
template <int C>
__device__ __forceinline__ int treduce32_lane(int c) {
  int lane = 0;
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const int half = (C >> s) >> 1;
    if (half >= 1 && (c & half)) lane |= (16 >> s);
  }
  return lane;
}

}  // namespace tsqr
