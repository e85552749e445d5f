// kernels_bitpacked.cu -- the bit-packed spin-1/2 layout: conversion to and
// from int8 spins, and (below) its sweep kernel.
//
// Layout: for colour c and row y, bit (j & 31) of word (j >> 5) holds the
// j-th colour-c site of the row (x = 2j + ((c + y) & 1)); a set bit is an
// up spin (+1).  Words per row bw = ceil((L/2) / 32).
#include "lattice_internal.cuh"

namespace lat {

namespace {

constexpr int kThreads = 256;

__global__ void k_pack(Geom g, const int8_t *s, uint32_t *bits)
{
    const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint64_t total = 2ull * g.L * g.bw;
    if (t >= total) return;
    const uint32_t k = (uint32_t)(t % g.bw);
    const uint32_t y = (uint32_t)((t / g.bw) % (uint64_t)g.L);
    const uint32_t c = (uint32_t)(t / ((uint64_t)g.bw * g.L));
    const uint32_t p = (c + y) & 1u;
    const uint32_t half = (uint32_t)g.L >> 1;
    uint32_t w = 0;
    for (uint32_t b = 0; b < 32; ++b) {
        const uint32_t j = 32 * k + b;
        if (j >= half) break;
        const uint32_t x = 2 * j + p;
        if (s[(uint64_t)y * g.L + x] > 0) w |= 1u << b;
    }
    bits[t] = w;
}

__global__ void k_unpack(Geom g, const uint32_t *bits, int8_t *s)
{
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= g.N) return;
    const uint32_t x = (uint32_t)(i % (uint64_t)g.L);
    const uint32_t y = (uint32_t)(i / (uint64_t)g.L);
    const uint32_t c = (x + y) & 1u;
    const uint32_t j = x >> 1;
    const uint32_t w = bits[((uint64_t)c * g.L + y) * g.bw + (j >> 5)];
    s[i] = ((w >> (j & 31)) & 1u) ? (int8_t)1 : (int8_t)-1;
}

}  // namespace

cudaError_t launch_pack_bits(const Geom &g, const int8_t *spins, uint32_t *bits, cudaStream_t st)
{
    const uint64_t total = 2ull * g.L * g.bw;
    k_pack<<<(unsigned)((total + kThreads - 1) / kThreads), kThreads, 0, st>>>(g, spins, bits);
    return cudaGetLastError();
}

cudaError_t launch_unpack_bits(const Geom &g, const uint32_t *bits, int8_t *spins, cudaStream_t st)
{
    k_unpack<<<(unsigned)((g.N + kThreads - 1) / kThreads), kThreads, 0, st>>>(g, bits, spins);
    return cudaGetLastError();
}

cudaError_t launch_sweep_bitpacked(const Geom &, int, cudaStream_t) { return cudaErrorNotSupported; }

}  // namespace lat
