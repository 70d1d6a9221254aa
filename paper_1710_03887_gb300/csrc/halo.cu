// Halo exchange of a partitioned mesh: the face traces of cut faces.
//
// A rank holds its own elements followed by copies of the neighbours' elements
// across its cut faces (halo elements). Every stage reads, of a halo element,
// only the nodes of the face it shares with an own element (the neighbour
// trace of Eq. 10's surface term), so an exchange moves 5 Nfp values per cut
// face: pack gathers them from own elements into a contiguous buffer
// [n][5][Nfp], the caller moves the buffer to the neighbour rank, and unpack
// scatters a received buffer into the halo elements' face nodes.
#include "dg_device.cuh"

namespace dgk {

namespace {

// ef[i] = e * 4 + f: element and face of entry i; buffer entry (i, v, m) is
// node Fmask[f][m] of variable v of element e
template <typename T>
__global__ void halo_pack_kernel(const T* __restrict__ q, int Np, int Nfp,
                                 const int32_t* __restrict__ ef, const int32_t* __restrict__ fmask,
                                 int64_t n, T* __restrict__ buf, int64_t K_all, int* status) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n * 5 * Nfp) return;
  const int64_t k = i / (5 * Nfp);
  const int r = int(i - k * 5 * Nfp), v = r / Nfp, m = r - (r / Nfp) * Nfp;
  const int32_t w = ef[k];
  const int64_t e = w >> 2;
  const int f = w & 3;
  const int node = fmask[f * Nfp + m];
  if (!DG_IN(e >= 0 && e < K_all && node >= 0 && node < Np, status)) return;
  buf[i] = q[(e * 5 + v) * Np + node];
}

template <typename T>
__global__ void halo_unpack_kernel(T* __restrict__ q, int Np, int Nfp,
                                   const int32_t* __restrict__ ef, const int32_t* __restrict__ fmask,
                                   int64_t n, const T* __restrict__ buf, int64_t K_all, int* status) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n * 5 * Nfp) return;
  const int64_t k = i / (5 * Nfp);
  const int r = int(i - k * 5 * Nfp), v = r / Nfp, m = r - (r / Nfp) * Nfp;
  const int32_t w = ef[k];
  const int64_t e = w >> 2;
  const int f = w & 3;
  const int node = fmask[f * Nfp + m];
  if (!DG_IN(e >= 0 && e < K_all && node >= 0 && node < Np, status)) return;
  q[(e * 5 + v) * Np + node] = buf[i];
}

}  // namespace

template <typename T>
cudaError_t launch_halo_pack(const T* q, int Np, int Nfp, const int32_t* ef, const int32_t* fmask,
                             int64_t n, T* buf, int64_t K_all, int* status, cudaStream_t s) {
  const int64_t total = n * 5 * Nfp;
  if (total == 0) return cudaSuccess;
  halo_pack_kernel<T><<<unsigned((total + 255) / 256), 256, 0, s>>>(q, Np, Nfp, ef, fmask, n, buf,
                                                                     K_all, status);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_halo_unpack(T* q, int Np, int Nfp, const int32_t* ef, const int32_t* fmask,
                               int64_t n, const T* buf, int64_t K_all, int* status, cudaStream_t s) {
  const int64_t total = n * 5 * Nfp;
  if (total == 0) return cudaSuccess;
  halo_unpack_kernel<T><<<unsigned((total + 255) / 256), 256, 0, s>>>(q, Np, Nfp, ef, fmask, n, buf,
                                                                       K_all, status);
  return cudaGetLastError();
}

template cudaError_t launch_halo_pack<float>(const float*, int, int, const int32_t*, const int32_t*,
                                             int64_t, float*, int64_t, int*, cudaStream_t);
template cudaError_t launch_halo_pack<double>(const double*, int, int, const int32_t*,
                                              const int32_t*, int64_t, double*, int64_t, int*,
                                              cudaStream_t);
template cudaError_t launch_halo_unpack<float>(float*, int, int, const int32_t*, const int32_t*,
                                               int64_t, const float*, int64_t, int*, cudaStream_t);
template cudaError_t launch_halo_unpack<double>(double*, int, int, const int32_t*, const int32_t*,
                                                int64_t, const double*, int64_t, int*, cudaStream_t);

}  // namespace dgk
