// Vertex-set bitsets used as wavefront states, for the three width classes of
// the expansion kernels: 32-bit (n <= 32), 64-bit (n <= 64) and 128-bit
// (n <= 128).  A state S is the set of eliminated vertices (arXiv 1709.09990,
// Section 3.1: the lists hold sets S of vertices with a feasible partial
// elimination ordering); bit v of the key is set iff v is in S.
#pragma once

#include <cstdint>

namespace tw {

struct K128 {
  unsigned long long lo, hi;
};

__host__ __device__ __forceinline__ K128 operator&(K128 a, K128 b) { return {a.lo & b.lo, a.hi & b.hi}; }
__host__ __device__ __forceinline__ K128 operator|(K128 a, K128 b) { return {a.lo | b.lo, a.hi | b.hi}; }
__host__ __device__ __forceinline__ K128 operator~(K128 a) { return {~a.lo, ~a.hi}; }
__host__ __device__ __forceinline__ bool operator==(K128 a, K128 b) { return a.lo == b.lo && a.hi == b.hi; }
__host__ __device__ __forceinline__ bool operator!=(K128 a, K128 b) { return !(a == b); }
__host__ __device__ __forceinline__ K128& operator|=(K128& a, K128 b) { a = a | b; return a; }
__host__ __device__ __forceinline__ K128& operator&=(K128& a, K128 b) { a = a & b; return a; }
__host__ __device__ __forceinline__ K128 operator^(K128 a, K128 b) { return {a.lo ^ b.lo, a.hi ^ b.hi}; }
__host__ __device__ __forceinline__ K128& operator^=(K128& a, K128 b) { a = a ^ b; return a; }

template <class K> struct KeyTraits;
template <> struct KeyTraits<uint32_t> { static constexpr int kBits = 32; static constexpr int kWords64 = 1; };
template <> struct KeyTraits<unsigned long long> { static constexpr int kBits = 64; static constexpr int kWords64 = 1; };
template <> struct KeyTraits<K128> { static constexpr int kBits = 128; static constexpr int kWords64 = 2; };

// ---- construction ---------------------------------------------------------
template <class K> __host__ __device__ __forceinline__ K kzero();
template <> __host__ __device__ __forceinline__ uint32_t kzero<uint32_t>() { return 0u; }
template <> __host__ __device__ __forceinline__ unsigned long long kzero<unsigned long long>() { return 0ull; }
template <> __host__ __device__ __forceinline__ K128 kzero<K128>() { return {0ull, 0ull}; }

template <class K> __host__ __device__ __forceinline__ K kones();
template <> __host__ __device__ __forceinline__ uint32_t kones<uint32_t>() { return ~0u; }
template <> __host__ __device__ __forceinline__ unsigned long long kones<unsigned long long>() { return ~0ull; }
template <> __host__ __device__ __forceinline__ K128 kones<K128>() { return {~0ull, ~0ull}; }

template <class K> __host__ __device__ __forceinline__ K kbit(int v);
template <> __host__ __device__ __forceinline__ uint32_t kbit<uint32_t>(int v) { return 1u << v; }
template <> __host__ __device__ __forceinline__ unsigned long long kbit<unsigned long long>(int v) { return 1ull << v; }
template <> __host__ __device__ __forceinline__ K128 kbit<K128>(int v) {
  return v < 64 ? K128{1ull << v, 0ull} : K128{0ull, 1ull << (v - 64)};
}

// The set {0, .., n-1}.
template <class K> __host__ __device__ __forceinline__ K kfirst_n(int n);
template <> __host__ __device__ __forceinline__ uint32_t kfirst_n<uint32_t>(int n) { return n >= 32 ? ~0u : ((1u << n) - 1u); }
template <> __host__ __device__ __forceinline__ unsigned long long kfirst_n<unsigned long long>(int n) {
  return n >= 64 ? ~0ull : ((1ull << n) - 1ull);
}
template <> __host__ __device__ __forceinline__ K128 kfirst_n<K128>(int n) {
  if (n >= 128) return {~0ull, ~0ull};
  if (n >= 64) return {~0ull, (n == 64) ? 0ull : ((1ull << (n - 64)) - 1ull)};
  return {(1ull << n) - 1ull, 0ull};
}

// ---- queries ----------------------------------------------------------------
__device__ __forceinline__ int kpopc(uint32_t a) { return __popc(a); }
__device__ __forceinline__ int kpopc(unsigned long long a) { return __popcll(a); }
__device__ __forceinline__ int kpopc(K128 a) { return __popcll(a.lo) + __popcll(a.hi); }

__host__ __device__ __forceinline__ bool kempty(uint32_t a) { return a == 0u; }
__host__ __device__ __forceinline__ bool kempty(unsigned long long a) { return a == 0ull; }
__host__ __device__ __forceinline__ bool kempty(K128 a) { return (a.lo | a.hi) == 0ull; }

// Index of the lowest set bit; the argument must be non-empty.
__device__ __forceinline__ int klowest(uint32_t a) { return __ffs(a) - 1; }
__device__ __forceinline__ int klowest(unsigned long long a) { return __ffsll(a) - 1; }
__device__ __forceinline__ int klowest(K128 a) { return a.lo ? __ffsll(a.lo) - 1 : 63 + __ffsll(a.hi); }

// a without its lowest set bit.
__device__ __forceinline__ uint32_t kdrop_lowest(uint32_t a) { return a & (a - 1u); }
__device__ __forceinline__ unsigned long long kdrop_lowest(unsigned long long a) { return a & (a - 1ull); }
__device__ __forceinline__ K128 kdrop_lowest(K128 a) {
  return a.lo ? K128{a.lo & (a.lo - 1ull), a.hi} : K128{0ull, a.hi & (a.hi - 1ull)};
}

// Lowest set bit of a as a one-bit set (a must be non-empty for an index).
__device__ __forceinline__ uint32_t klsb(uint32_t a) { return a & (0u - a); }
__device__ __forceinline__ unsigned long long klsb(unsigned long long a) { return a & (0ull - a); }
__device__ __forceinline__ K128 klsb(K128 a) {
  return a.lo ? K128{a.lo & (0ull - a.lo), 0ull} : K128{0ull, a.hi & (0ull - a.hi)};
}

// The vertices below the lowest element of a (every vertex when a is empty).
__device__ __forceinline__ uint32_t kbelow_lowest(uint32_t a) { return (a - 1u) & ~a; }
__device__ __forceinline__ unsigned long long kbelow_lowest(unsigned long long a) { return (a - 1ull) & ~a; }
__device__ __forceinline__ K128 kbelow_lowest(K128 a) {
  return a.lo ? K128{(a.lo - 1ull) & ~a.lo, 0ull} : K128{~0ull, (a.hi - 1ull) & ~a.hi};
}

// Index of the only set bit of a one-bit set.
__device__ __forceinline__ int kindex(uint32_t b) { return 31 - __clz(b); }
__device__ __forceinline__ int kindex(unsigned long long b) { return 63 - __clzll(b); }
__device__ __forceinline__ int kindex(K128 b) { return b.lo ? 63 - __clzll(b.lo) : 127 - __clzll(b.hi); }

__device__ __forceinline__ bool ktest(uint32_t a, int v) { return (a >> v) & 1u; }
__device__ __forceinline__ bool ktest(unsigned long long a, int v) { return (a >> v) & 1ull; }
__device__ __forceinline__ bool ktest(K128 a, int v) { return v < 64 ? ((a.lo >> v) & 1ull) : ((a.hi >> (v - 64)) & 1ull); }

// Warp shuffle of a key from lane src.
__device__ __forceinline__ uint32_t kshfl(uint32_t a, int src) { return __shfl_sync(0xffffffffu, a, src); }
__device__ __forceinline__ unsigned long long kshfl(unsigned long long a, int src) {
  return __shfl_sync(0xffffffffu, a, src);
}
__device__ __forceinline__ K128 kshfl(K128 a, int src) {
  return K128{__shfl_sync(0xffffffffu, a.lo, src), __shfl_sync(0xffffffffu, a.hi, src)};
}

// ---- hashing ----------------------------------------------------------------
// 64-bit finaliser of MurmurHash3 (Appleby); the paper also hashes states with
// Murmur3 (Section 3.2).
__host__ __device__ __forceinline__ unsigned long long fmix64(unsigned long long x) {
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdull;
  x ^= x >> 33;
  x *= 0xc4ceb9fe1a85ec53ull;
  x ^= x >> 33;
  return x;
}
__device__ __forceinline__ unsigned long long khash(uint32_t a) { return fmix64((unsigned long long)a); }
__device__ __forceinline__ unsigned long long khash(unsigned long long a) { return fmix64(a); }
__device__ __forceinline__ unsigned long long khash(K128 a) { return fmix64(a.lo ^ fmix64(a.hi ^ 0x9e3779b97f4a7c15ull)); }

// Level fingerprint fp(S) = mix(w0 ^ mix(w1)) with mix the splitmix64 output
// function (Steele, Lea & Flood 2014).  Order independent once summed.
__device__ __forceinline__ unsigned long long splitmix_out(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ unsigned long long kfingerprint(uint32_t a) { return splitmix_out((unsigned long long)a ^ splitmix_out(0ull)); }
__device__ __forceinline__ unsigned long long kfingerprint(unsigned long long a) { return splitmix_out(a ^ splitmix_out(0ull)); }
__device__ __forceinline__ unsigned long long kfingerprint(K128 a) { return splitmix_out(a.lo ^ splitmix_out(a.hi)); }

// ---- atomics ----------------------------------------------------------------
__device__ __forceinline__ uint32_t kcas(uint32_t* p, uint32_t cmp, uint32_t val) {
  return atomicCAS(reinterpret_cast<unsigned int*>(p), cmp, val);
}
__device__ __forceinline__ unsigned long long kcas(unsigned long long* p, unsigned long long cmp,
                                                   unsigned long long val) {
  return atomicCAS(p, cmp, val);
}
// 16-byte compare-and-swap (PTX atom.cas.b128, sm_90 and later); p must be
// 16-byte aligned.
__device__ __forceinline__ K128 kcas(K128* p, K128 cmp, K128 val) {
  K128 old;
  asm volatile(
      "{\n\t.reg .b128 c, v, o;\n\t"
      "mov.b128 c, {%2, %3};\n\t"
      "mov.b128 v, {%4, %5};\n\t"
      "atom.global.cas.b128 o, [%6], c, v;\n\t"
      "mov.b128 {%0, %1}, o;\n\t}"
      : "=l"(old.lo), "=l"(old.hi)
      : "l"(cmp.lo), "l"(cmp.hi), "l"(val.lo), "l"(val.hi), "l"(p)
      : "memory");
  return old;
}

// Load that bypasses L1 (the table is written by other SMs during a level).
__device__ __forceinline__ uint32_t kload_cg(const uint32_t* p) { return __ldcg(p); }
__device__ __forceinline__ unsigned long long kload_cg(const unsigned long long* p) { return __ldcg(p); }
__device__ __forceinline__ K128 kload_cg(const K128* p) {
  ulonglong2 v = __ldcg(reinterpret_cast<const ulonglong2*>(p));
  return {v.x, v.y};
}

// Streaming (evict-first) load and store for the level lists, which are read
// or written once per level, so that the hash table keeps the L2.
__device__ __forceinline__ uint32_t kload_cs(const uint32_t* p) { return __ldcs(p); }
__device__ __forceinline__ unsigned long long kload_cs(const unsigned long long* p) { return __ldcs(p); }
__device__ __forceinline__ K128 kload_cs(const K128* p) {
  const ulonglong2 v = __ldcs(reinterpret_cast<const ulonglong2*>(p));
  return {v.x, v.y};
}
__device__ __forceinline__ void kstore_cs(uint32_t* p, uint32_t v) { __stcs(p, v); }
__device__ __forceinline__ void kstore_cs(unsigned long long* p, unsigned long long v) { __stcs(p, v); }
__device__ __forceinline__ void kstore_cs(K128* p, K128 v) {
  __stcs(reinterpret_cast<ulonglong2*>(p), make_ulonglong2(v.lo, v.hi));
}

}  // namespace tw
