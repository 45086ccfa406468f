// Counter-based Gaussian numbers: splitmix64 (Steele, Lea & Flood, "Fast
// splittable pseudorandom number generators", OOPSLA 2014) of a 64-bit key,
// turned into two normals by the Box-Muller transform.
#pragma once

namespace ce {

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// key of element (row g, column c) of the sketch of block i at a level
__device__ __forceinline__ unsigned long long sketch_key(unsigned long long seed, int level, int i,
                                                         int g, int c) {
  return splitmix64(seed ^ splitmix64(((unsigned long long)level << 48) ^ ((unsigned long long)i << 24) ^
                                      (unsigned long long)(g * 128 + c)));
}

// N(0, 1) from a 64-bit key (two 32-bit uniforms, Box-Muller cosine branch)
__device__ __forceinline__ float gauss_from_key(unsigned long long k) {
  const float u1 = ((float)(k >> 40) + 1.0f) * (1.0f / 16777217.0f);
  const float u2 = (float)((k >> 8) & 0xFFFFFFull) * (1.0f / 16777216.0f);
  return sqrtf(-2.0f * __logf(u1)) * __cosf(6.2831853071795865f * u2);
}

}  // namespace ce
