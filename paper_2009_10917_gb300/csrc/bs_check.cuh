// Device-side index checks of the checked build (-DBS_CHECK=1).
//
// In a checked build every kernel tests each index it takes from memory with
// the predicates of bs_check_pred.h before using it: a failing test records
// its code in this translation unit's check word (the first failure wins)
// and the access is skipped (a load reads 0, a store is dropped), so bad data
// never reaches memory outside the buffers.  Each unit registers a reader of
// its word at load time; bs_check_device() waits for the device, collects
// and clears the words of all units and reports the first code.  In the
// default build chk() is the constant true and the tests compile away.
#pragma once

#include <cuda_runtime.h>

#include "bs_check_pred.h"

#ifndef BS_CHECK
#define BS_CHECK 0
#endif

namespace bs {

// Registers a reader of one unit's check word (bs_core.cu); the reader
// stores the word and clears it, returning 0 or -1 on a CUDA error.
int register_check_word(int (*read_and_clear)(unsigned int *));

#if BS_CHECK
namespace {
__device__ unsigned int tu_check_word;

int tu_check_read_and_clear(unsigned int *out) {
  const unsigned int zero = 0;
  *out = 0;
  if (cudaMemcpyFromSymbol(out, tu_check_word, sizeof(unsigned int)) != cudaSuccess) return -1;
  if (*out && cudaMemcpyToSymbol(tu_check_word, &zero, sizeof zero) != cudaSuccess) return -1;
  return 0;
}

const int tu_check_registered = register_check_word(&tu_check_read_and_clear);
}  // namespace

// ok, after recording `code` when it is false.
__device__ __forceinline__ bool chk(bool ok, unsigned int code) {
  if (!ok) atomicCAS(&tu_check_word, 0u, code);
  return ok;
}
#else
__device__ __forceinline__ constexpr bool chk(bool, unsigned int) { return true; }
#endif

}  // namespace bs
