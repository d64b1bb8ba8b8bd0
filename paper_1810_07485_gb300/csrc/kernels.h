// Launch interface between the host engine and the update kernels.
#pragma once
#include "dev.cuh"

namespace lcq {

// One batch's launch geometry.  Tiles, site blocks and bond blocks are ordered
// with every Q=1 chain's blocks before every Q=2 chain's blocks; index [q]
// addresses the Q = q+1 group.
struct Launch {
  DevChain *ch;
  int nchains;
  Scratch s;
  const int2 *tile_tab, *site_tab, *bond_tab;
  int64_t ntile[2], tile0[2];
  int64_t nsiteblk[2], site0[2];
  int64_t nbondblk[2], bond0[2];
  int temporal;  // measure the temporal moment chi(pi, 2 pi / beta) too
};

void set_full_table(const uint64_t *T, cudaStream_t st);
int init_kernel_attributes();
void launch_bond_parity(const Launch &L, cudaStream_t st);
void launch_insert(const Launch &L, cudaStream_t st);
void launch_scan_ops(const Launch &L, cudaStream_t st);
void launch_cut(const Launch &L, cudaStream_t st);
void launch_link(const Launch &L, cudaStream_t st);
void launch_compress(const Launch &L, cudaStream_t st);
void launch_est(const Launch &L, cudaStream_t st);
void launch_compact(const Launch &L, cudaStream_t st);
void launch_sites(const Launch &L, cudaStream_t st);
void launch_final(const Launch &L, cudaStream_t st);

}  // namespace lcq
