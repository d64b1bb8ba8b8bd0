// Lock-free union-find on int32 node ids (device functions).
#pragma once
#include <cstdint>

#include "dev.cuh"

namespace lcq {

// ---- union-find (Sec. 3.2): min-root hooking with one CAS --------------------
// parent[x] <= x always holds; a root is its own parent.  A link is made by a
// single compare-and-swap on the larger root's parent word, which both checks
// that it is still a root and attaches it: the lock of steps 4'-6' and the
// pointer update in one instruction, with no weight kept.
// limit: the most steps a walk or a retry loop may take (UF_MAX_ITERS unless
// a test lowers it); past it the status word gets ST_TIMEOUT and the call
// returns early (every later kernel of the update then stops at entry).
__device__ inline int uf_find(int32_t *par, int x, int *status, int limit = UF_MAX_ITERS) {
  int p = __ldcg(par + x);
  if (p == x) return x;
  int prev = x;
  for (int it = 0;; ++it) {
    int next = __ldcg(par + p);
    if (next >= p) break;
    par[prev] = next;  // path halving: skip one level
    prev = p;
    p = next;
    if (it >= limit) {
      atomicOr(status, ST_TIMEOUT);
      break;
    }
  }
  return p;
}

// Read-only walk to the root.  Compression uses it so that the only store to
// parent[v] in that phase is v's own root: a path-halving store from another
// thread landing after it would leave a non-root ancestor behind.
__device__ inline int uf_root(const int32_t *par, int x, int *status, int limit = UF_MAX_ITERS) {
  int p = __ldcg(par + x);
  for (int it = 0; p != x; ++it) {
    x = p;
    p = __ldcg(par + x);
    if (it >= limit) {
      atomicOr(status, ST_TIMEOUT);
      break;
    }
  }
  return x;
}

__device__ inline void uf_union(int32_t *par, int a, int b, int *status, int limit = UF_MAX_ITERS) {
  a = uf_find(par, a, status, limit);
  b = uf_find(par, b, status, limit);
  for (int it = 0; it < limit; ++it) {
    if (a == b) return;
    if (a > b) {
      int t = a;
      a = b;
      b = t;
    }
    int old = atomicCAS(par + b, b, a);
    if (old == b) return;
    b = old;  // b was attached meanwhile: continue from its new parent
  }
  atomicOr(status, ST_TIMEOUT);
}

}  // namespace lcq
