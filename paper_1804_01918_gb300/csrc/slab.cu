// slab.cu -- ghost-row exchange of a lattice cut into horizontal slabs (one slab per GPU, or
// several per GPU), the domain decomposition of the multi-GPU path.
//
// The paper runs one KNL socket and names a hybrid MPI + OpenMP code over many nodes as future
// work (Sec. 5). Because every site of a step depends only on sites at most three rows away (the
// D2Q37 pull reaches |c_y| <= 3, Sec. 3), a lattice cut along y into slabs needs, per step and per
// cut, only the populations that cross the cut: a slab's ghost row k below its row 0 (k = 1, 2, 3)
// is read by the pull only for populations with c_y >= k, i.e. 15 + 8 + 3 = 26 population-rows,
// and symmetrically 26 above (c_y <= -k). x stays periodic inside every slab.
//
// Ghost-row order, shared by pack, unpack and the in-process exchange (GhostRows below): k = 1, 2,
// 3 outward from the cut, and for each k the populations in the library's order whose velocity
// crosses the cut by at least k rows. Each entry is one row of Lx elements.
#include <cuda_runtime.h>

#include <cstdint>

#include "d2q37_gpu.cuh"
#include "kernels.cuh"

namespace lbg {

namespace {

// The 26 (population, k) entries of one direction: up = populations moving up (c_y >= k), which a
// slab receives below its row 0 and sends from its top rows; down = c_y <= -k.
struct GhostRows {
    int n;
    int pop[26];
    int k[26];
};

GhostRows ghost_rows(bool up) {
    GhostRows g{};
    for (int k = 1; k <= HALO; ++k)
        for (int i = 0; i < NPOP; ++i) {
            const int c = up ? cy_of(i) : -cy_of(i);
            if (c >= k) {
                g.pop[g.n] = i;
                g.k[g.n] = k;
                ++g.n;
            }
        }
    return g;
}

// Padded row (0 .. Ly + 5) of entry j: the sent row is the k-th row inward from the cut, the ghost
// row the k-th row outward. side 0 = the cut below row 0, side 1 = the cut above row Ly - 1.
__host__ __device__ inline int sent_row(int side, int k, int Ly) { return side == 0 ? HALO + k - 1 : HALO + Ly - k; }
__host__ __device__ inline int ghost_row(int side, int k, int Ly) { return side == 0 ? HALO - k : HALO + Ly - 1 + k; }

// Rows of one direction copied element by element: entry j = blockIdx.y, x = grid-stride over Lx.
// mode 0: lattice -> packed buffer (pack), 1: packed buffer -> lattice (unpack), 2: lattice ->
// lattice (in-process exchange).
template <typename T>
__global__ void ghost_copy_kernel(const T* __restrict__ a, T* __restrict__ b, GhostRows g, int mode,
                                  int Lx, long long plane_a, long long plane_b, int row_a_side, int Ly_a,
                                  int row_b_side, int Ly_b) {
    const int j = blockIdx.y;
    if (j >= g.n) return;
    const int i = g.pop[j], k = g.k[j];
    long long oa, ob;
    if (mode == 0) {  // a: lattice (sent row), b: buffer row j
        oa = (long long)i * plane_a + (long long)sent_row(row_a_side, k, Ly_a) * Lx;
        ob = (long long)j * Lx;
    } else if (mode == 1) {  // a: buffer row j, b: lattice (ghost row)
        oa = (long long)j * Lx;
        ob = (long long)i * plane_b + (long long)ghost_row(row_b_side, k, Ly_b) * Lx;
    } else {  // a: sending lattice, b: receiving lattice
        oa = (long long)i * plane_a + (long long)sent_row(row_a_side, k, Ly_a) * Lx;
        ob = (long long)i * plane_b + (long long)ghost_row(row_b_side, k, Ly_b) * Lx;
    }
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < Lx; x += gridDim.x * blockDim.x)
        b[ob + x] = a[oa + x];
}

template <typename T>
cudaError_t ghost_copy(const void* a, void* b, bool up, int mode, int Lx, long long plane_a, long long plane_b,
                       int side_a, int Ly_a, int side_b, int Ly_b, cudaStream_t s) {
    const GhostRows g = ghost_rows(up);
    const dim3 grid((unsigned)((Lx + 255) / 256), (unsigned)g.n);
    ghost_copy_kernel<T><<<grid, 256, 0, s>>>((const T*)a, (T*)b, g, mode, Lx, plane_a, plane_b, side_a, Ly_a,
                                              side_b, Ly_b);
    return cudaGetLastError();
}

cudaError_t ghost_copy_any(size_t elem, const void* a, void* b, bool up, int mode, int Lx, long long plane_a,
                           long long plane_b, int side_a, int Ly_a, int side_b, int Ly_b, cudaStream_t s) {
    return elem == 8 ? ghost_copy<double>(a, b, up, mode, Lx, plane_a, plane_b, side_a, Ly_a, side_b, Ly_b, s)
                     : ghost_copy<float>(a, b, up, mode, Lx, plane_a, plane_b, side_a, Ly_a, side_b, Ly_b, s);
}

}  // namespace

int ghost_row_count() { return ghost_rows(true).n; }

// Pack the rows a slab sends across its cut `side` (0 below, 1 above) from lattice f into buf
// [26][Lx]: across the cut below go the populations moving down (c_y <= -k), above those moving up.
cudaError_t launch_slab_pack(size_t elem, const void* f, void* buf, const StepParams& P, int side, cudaStream_t s) {
    return ghost_copy_any(elem, f, buf, side == 1, 0, P.Lx, P.plane, 0, side, P.Ly, 0, 0, s);
}

// Unpack buf [26][Lx] (what the neighbour across `side` sent) into the ghost rows of f at `side`:
// below row 0 arrive the populations moving up, above row Ly - 1 those moving down.
cudaError_t launch_slab_unpack(size_t elem, const void* buf, void* f, const StepParams& P, int side,
                               cudaStream_t s) {
    return ghost_copy_any(elem, buf, f, side == 0, 1, P.Lx, 0, P.plane, 0, 0, side, P.Ly, s);
}

// Exchange across the cut between slab `lo` (below) and slab `hi` (above), lattice to lattice:
// lo's top rows -> hi's ghost rows below (populations moving up), hi's bottom rows -> lo's ghost
// rows above (populations moving down).
cudaError_t launch_slab_exchange(size_t elem, void* f_lo, const StepParams& Plo, void* f_hi,
                                 const StepParams& Phi, cudaStream_t s) {
    cudaError_t e = ghost_copy_any(elem, f_lo, f_hi, true, 2, Plo.Lx, Plo.plane, Phi.plane, 1, Plo.Ly, 0,
                                   Phi.Ly, s);
    if (e != cudaSuccess) return e;
    return ghost_copy_any(elem, f_hi, f_lo, false, 2, Plo.Lx, Phi.plane, Plo.plane, 0, Phi.Ly, 1, Plo.Ly, s);
}

}  // namespace lbg
