// Host-memory stand-ins for the few CUDA runtime calls the batched plan code makes,
// so that its host logic can run on a CPU under AddressSanitizer (test only).
#pragma once
#include <cstdlib>
#include <cstring>
#include <cstdint>
typedef int cudaError_t; enum { cudaSuccess = 0, cudaErrorInvalidValue = 1 };
typedef void* cudaStream_t;
enum cudaMemcpyKind { cudaMemcpyHostToDevice, cudaMemcpyDeviceToDevice, cudaMemcpyDeviceToHost };
enum { cudaDevAttrMultiProcessorCount };
struct float2 { float x, y; };
inline cudaError_t cudaMalloc(void* p, size_t n) { *(void**)p = malloc(n); return 0; }
template <class T> inline cudaError_t cudaMalloc(T** p, size_t n) { *p = (T*)malloc(n); return 0; }
inline cudaError_t cudaFree(void* p) { free(p); return 0; }
inline cudaError_t cudaMemcpy(void* d, const void* s, size_t n, cudaMemcpyKind) { memcpy(d, s, n); return 0; }
inline cudaError_t cudaMemset(void* d, int v, size_t n) { memset(d, v, n); return 0; }
inline cudaError_t cudaGetDevice(int* d) { *d = 0; return 0; }
inline cudaError_t cudaDeviceGetAttribute(int* v, int, int) { *v = 152; return 0; }
inline cudaError_t cudaDeviceSynchronize() { return 0; }
inline cudaError_t cudaStreamSynchronize(cudaStream_t) { return 0; }
#define __host__
#define __device__
#define __forceinline__ inline
