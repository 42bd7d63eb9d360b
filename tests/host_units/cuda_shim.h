// Declarations that let the library's device helper headers compile as plain host C++ for
// the CPU unit tests of their scalar functions. Only declared, never defined: a scalar test
// that reached a warp-collective helper would fail to link. (The warp- and block-collective
// helpers are tested on the SIMT emulator of simt_emu.h instead.)
#pragma once
struct gbfs_host_dim3 {
  unsigned x, y, z;
};
extern gbfs_host_dim3 threadIdx, blockIdx, blockDim, gridDim;
unsigned __ldcg(const unsigned*);
unsigned __ballot_sync(unsigned, int);
int __ffs(unsigned);
int __popc(unsigned);
template <class T>
T __shfl_sync(unsigned, T, int);
template <class T>
T __shfl_up_sync(unsigned, T, unsigned);
void __syncthreads();
