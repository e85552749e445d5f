// kernels_bitpacked.cu -- the bit-packed spin-1/2 layout: conversion to and
// from int8 spins, and (below) its sweep kernel.
//
// Layout: for colour c and row y, bit (j & 31) of word (j >> 5) holds the
// j-th colour-c site of the row (x = 2j + ((c + y) & 1)), i.e. entry j of
// row y of colour plane c of the planar int8 layout; a set bit is an up
// spin (+1).  Words per row bw = ceil((L/2) / 32).
#include "lattice_internal.cuh"

namespace lat {

namespace {

constexpr int kThreads = 256;

// planar int8 -> bits: word k of plane c row y holds sites j = 32k .. 32k+31.
__global__ void k_pack(Geom g, const int8_t *planar, uint32_t *bits)
{
    const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint64_t total = 2ull * g.L * g.bw;
    if (t >= total) return;
    const uint32_t k = (uint32_t)(t % g.bw);
    const uint64_t row = t / g.bw;  // c * L + y
    const int8_t *src = planar + row * g.half;
    uint32_t w = 0;
    for (uint32_t b = 0; b < 32; ++b) {
        const uint32_t j = 32 * k + b;
        if (j >= g.half) break;
        if (src[j] > 0) w |= 1u << b;
    }
    bits[t] = w;
}

__global__ void k_unpack(Geom g, const uint32_t *bits, int8_t *planar)
{
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= g.N) return;
    const uint64_t row = i / g.half;  // c * L + y
    const uint32_t j = (uint32_t)(i % g.half);
    const uint32_t w = bits[row * g.bw + (j >> 5)];
    planar[i] = ((w >> (j & 31)) & 1u) ? (int8_t)1 : (int8_t)-1;
}

}  // namespace

cudaError_t launch_pack_bits(const Geom &g, const int8_t *planar, uint32_t *bits, cudaStream_t st)
{
    const uint64_t total = 2ull * g.L * g.bw;
    k_pack<<<(unsigned)((total + kThreads - 1) / kThreads), kThreads, 0, st>>>(g, planar, bits);
    return cudaGetLastError();
}

cudaError_t launch_unpack_bits(const Geom &g, const uint32_t *bits, int8_t *planar, cudaStream_t st)
{
    k_unpack<<<(unsigned)((g.N + kThreads - 1) / kThreads), kThreads, 0, st>>>(g, bits, planar);
    return cudaGetLastError();
}

cudaError_t launch_sweep_bitpacked(const Geom &, int, cudaStream_t) { return cudaErrorNotSupported; }

}  // namespace lat
