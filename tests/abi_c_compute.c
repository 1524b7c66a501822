/* A plain C consumer of the compute calls (compiled and run by tests/test_abi_c.py on a GPU):
 * it includes only include/fpdqt.h and the CUDA runtime's C header, reads seeded inputs from
 * files the test wrote, copies them to device memory it allocates itself, runs a matrix
 * product, a batched polynomial product and a dot product through the C ABI on its own
 * stream, copies the results back and writes them to files for the test to compare with the
 * oracle.  Usage: abi_c_compute <dir> p m n k batch deg n_dot */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime_api.h>

#include "fpdqt.h"

static int read_file(const char* dir, const char* name, void* dst, size_t bytes) {
  char path[1024];
  snprintf(path, sizeof path, "%s/%s", dir, name);
  FILE* f = fopen(path, "rb");
  if (!f) return 1;
  const size_t got = fread(dst, 1, bytes, f);
  fclose(f);
  return got != bytes;
}

static int write_file(const char* dir, const char* name, const void* src, size_t bytes) {
  char path[1024];
  snprintf(path, sizeof path, "%s/%s", dir, name);
  FILE* f = fopen(path, "wb");
  if (!f) return 1;
  const size_t put = fwrite(src, 1, bytes, f);
  fclose(f);
  return put != bytes;
}

#define CK(x)                                                             \
  do {                                                                    \
    if ((x) != cudaSuccess) {                                             \
      fprintf(stderr, "CUDA call failed at line %d: %s\n", __LINE__, #x); \
      return 2;                                                           \
    }                                                                     \
  } while (0)

#define FK(x)                                                                           \
  do {                                                                                  \
    const fp_status s_ = (x);                                                           \
    if (s_ != FP_OK) {                                                                  \
      fprintf(stderr, "library call failed at line %d: %d %s\n", __LINE__, (int)s_,    \
              fp_last_error());                                                         \
      return 3;                                                                         \
    }                                                                                   \
  } while (0)

int main(int argc, char** argv) {
  if (argc != 9) {
    fprintf(stderr, "usage: %s dir p m n k batch deg n_dot\n", argv[0]);
    return 1;
  }
  const char* dir = argv[1];
  const uint32_t p = (uint32_t)atoi(argv[2]);
  const int m = atoi(argv[3]), n = atoi(argv[4]), k = atoi(argv[5]);
  const size_t batch = (size_t)atol(argv[6]);
  const uint32_t deg = (uint32_t)atoi(argv[7]);
  const size_t nd = (size_t)atol(argv[8]);
  const size_t sa = (size_t)m * k, sb = (size_t)k * n, sc = (size_t)m * n;
  const size_t spa = batch * (deg + 1), spc = batch * (2 * deg + 1);
  uint8_t* hA = malloc(sa);
  uint8_t* hB = malloc(sb);
  uint8_t* hC = malloc(sc);
  uint8_t* hPa = malloc(spa);
  uint8_t* hPb = malloc(spa);
  uint8_t* hPc = malloc(spc);
  uint8_t* hU = malloc(nd);
  uint8_t* hV = malloc(nd);
  if (!hA || !hB || !hC || !hPa || !hPb || !hPc || !hU || !hV) return 4;
  if (read_file(dir, "A.bin", hA, sa) || read_file(dir, "B.bin", hB, sb) || read_file(dir, "Pa.bin", hPa, spa) ||
      read_file(dir, "Pb.bin", hPb, spa) || read_file(dir, "U.bin", hU, nd) || read_file(dir, "V.bin", hV, nd)) {
    fprintf(stderr, "missing input file\n");
    return 5;
  }
  CK(cudaSetDevice(0));
  cudaStream_t st;
  CK(cudaStreamCreate(&st));
  uint8_t *dA, *dB, *dC, *dPa, *dPb, *dPc, *dU, *dV;
  uint32_t* dDot;
  CK(cudaMalloc((void**)&dA, sa));
  CK(cudaMalloc((void**)&dB, sb));
  CK(cudaMalloc((void**)&dC, sc));
  CK(cudaMalloc((void**)&dPa, spa));
  CK(cudaMalloc((void**)&dPb, spa));
  CK(cudaMalloc((void**)&dPc, spc));
  CK(cudaMalloc((void**)&dU, nd));
  CK(cudaMalloc((void**)&dV, nd));
  CK(cudaMalloc((void**)&dDot, sizeof(uint32_t)));
  CK(cudaMemcpyAsync(dA, hA, sa, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(dB, hB, sb, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(dPa, hPa, spa, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(dPb, hPb, spa, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(dU, hU, nd, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(dV, hV, nd, cudaMemcpyHostToDevice, st));

  fp_ctx ctx = NULL;
  FK(fp_ctx_create(&ctx, 0));
  FK(fp_matmul(ctx, p, m, n, k, dA, k, dB, n, dC, n, FP_MM_AUTO, (void*)st));
  FK(fp_polymul_batched(ctx, p, dPa, deg, dPb, deg, dPc, batch, FP_ALGO_AUTO, (void*)st));
  FK(fp_dot(ctx, p, dU, dV, nd, dDot, FP_ALGO_AUTO, (void*)st));
  FK(fp_ctx_status(ctx, (void*)st));
  uint32_t dot = 0;
  CK(cudaMemcpyAsync(hC, dC, sc, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(hPc, dPc, spc, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&dot, dDot, sizeof dot, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));

  /* a residue out of range is reported by the context status, not by a fault */
  const uint8_t bad = (uint8_t)p;
  CK(cudaMemcpy(dA, &bad, 1, cudaMemcpyHostToDevice));
  FK(fp_matmul(ctx, p, m, n, k, dA, k, dB, n, dC, n, FP_MM_AUTO, (void*)st));
  const fp_status range = fp_ctx_status(ctx, (void*)st);
  fp_ctx_destroy(ctx);

  if (write_file(dir, "C.bin", hC, sc) || write_file(dir, "Pc.bin", hPc, spc) ||
      write_file(dir, "dot.bin", &dot, sizeof dot))
    return 6;
  printf("range_status %d\n", (int)range);
  cudaFree(dA);
  cudaFree(dB);
  cudaFree(dC);
  cudaFree(dPa);
  cudaFree(dPb);
  cudaFree(dPc);
  cudaFree(dU);
  cudaFree(dV);
  cudaFree(dDot);
  cudaStreamDestroy(st);
  free(hA);
  free(hB);
  free(hC);
  free(hPa);
  free(hPb);
  free(hPc);
  free(hU);
  free(hV);
  return 0;
}
