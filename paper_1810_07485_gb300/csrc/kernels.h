// Launch interface between the host engine and the update kernels.
#pragma once
#include "dev.cuh"

namespace lcq {

// One batch's launch geometry.  Tiles, site blocks and bond blocks are grouped
// by Q = 2S (every Q=1 chain's blocks first, then Q=2, ...); index [q]
// addresses the Q = q+1 group.
struct Launch {
  DevChain *ch;
  int nchains;
  Scratch s;
  const int2 *tile_tab, *site_tab, *bond_tab;
  int64_t ntile[QMAX], tile0[QMAX];
  int64_t nsiteblk[QMAX], site0[QMAX];
  int64_t nbondblk[QMAX], bond0[QMAX];
  int temporal;  // measure the temporal moment chi(pi, 2 pi / beta) too
  // block sizes of the union-find phases (any choice gives the same results)
  int link_threads = 256;     // k_link: 128 or 256
  int link_x_warps = 8;       // k_link_x: 1 .. 8 warps (one tile each) per block
  int compress_threads = 128; // k_compress: 32, 64, 96 or 128
  int check_forest = 0;       // verify the loop forest after compression (debug)
};

void set_full_table(const uint64_t *T, cudaStream_t st);
int init_kernel_attributes();
void launch_bond_parity(const Launch &L, cudaStream_t st);
// zeroes the look-back words of ntile tiles, the tickets and nw words of each bitmap
void launch_clear(const Launch &L, int64_t ntile, int64_t nw, cudaStream_t st);
void launch_insert(const Launch &L, cudaStream_t st);
void launch_scan_ops(const Launch &L, cudaStream_t st);
void launch_cut(const Launch &L, cudaStream_t st);
void launch_link(const Launch &L, cudaStream_t st);
void launch_compress(const Launch &L, cudaStream_t st);
void launch_check_forest(const Launch &L, cudaStream_t st);
void launch_est(const Launch &L, cudaStream_t st);
void launch_compact(const Launch &L, cudaStream_t st);
void launch_sites(const Launch &L, cudaStream_t st);
void launch_final(const Launch &L, cudaStream_t st);

}  // namespace lcq
