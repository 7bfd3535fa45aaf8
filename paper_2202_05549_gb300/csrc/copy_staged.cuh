// Packs and write-backs through shared memory (declared apart from kernels.cuh,
// whose other kernels it does not touch).
#pragma once
#include "kernels.cuh"

namespace lt::k {
// copy_pieces through shared memory with bulk asynchronous copies (TMA, no
// tensor map) for units of whole rows whose 16-byte aligned body is equally
// aligned on both sides and fits the 64 KB stage; other units take the
// register path of copy_pieces.  A bounded wait that expires records 0x6730 in
// *err (the unit is then left uncopied, the launch's error word set).
cudaError_t copy_pieces_staged(const CopyPiece *dev, int n, uint64_t total_units, uint32_t *err, cudaStream_t st);
}  // namespace lt::k
