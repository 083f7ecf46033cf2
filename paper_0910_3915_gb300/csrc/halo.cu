// Face messages of a lattice decomposed into z slabs (the LB update needs
// only nearest neighbours, Sec. 2, so a slab needs one plane of each
// neighbour per step).
//
// A slab owns planes 1..nz-2 of its context; plane 0 and plane nz-1 are halo
// planes where it has a neighbour (else the solid wall layers). A step
// pushes the slab's populations into its halo planes like into fluid nodes.
// After the step, for the face between a slab A below and B above:
//   - the 5 populations per component that A pushed across (c_z = +1, into
//     A's top halo plane) belong to B's first owned plane, and the 5 that B
//     pushed down (c_z = -1, into B's bottom halo plane) to A's last owned plane;
//   - B's bottom halo plane must become A's last owned plane: its 14 slots per
//     component with c_z >= 0 are final in A after A's step, and its c_z = -1
//     slots are the very values B just pushed into that halo plane itself
//     (symmetrically for A's top halo plane).
// So each face message carries 38 planes of nx*ny values: entries 0..9 the
// crossing populations (component a, i-th velocity of the crossing set:
// entry a*5 + i), entries 10..37 the boundary plane's 14 slots per component
// with c_z of the message's direction or 0 (entry 10 + a*14 + i). Values
// travel in their storage format, x fastest, then y: a copy, no arithmetic.
#include "lb_fields.cuh"

namespace lbsc {

// velocity of the i-th member of the set crossing in direction dir (+1: up, -1: down)
__device__ __forceinline__ int cross_k(int i, int dir)
{
    // c_z = +1: (0,0,1), (1,0,1), (-1,0,1), (0,1,1), (0,-1,1); c_z = -1: their opposites
    const int up = i == 0 ? 5 : (i == 1 ? 11 : (i == 2 ? 14 : (i == 3 ? 15 : 18)));
    return dir > 0 ? up : opp(up);
}
// i-th of the 14 slots with c_z in {0, dir}: the 9 with c_z = 0, then the crossing set
__device__ __forceinline__ int plane_k(int i, int dir)
{
    if (i < 9) return i < 5 ? i : i + 2;  // 0..4 (rest, +-x, +-y), 7..10 (the xy diagonals)
    return cross_k(i - 9, dir);
}
// component a, velocity k and plane z of message entry j for a face whose
// crossing entries live on plane zc with direction dc and whose plane entries
// live on plane zp with direction dp
__device__ __forceinline__ void entry_of(int j, int zc, int dc, int zp, int dp, int& a, int& k, int& z)
{
    if (j < 10) {
        a = j / 5;
        k = cross_k(j % 5, dc);
        z = zc;
    } else {
        const int t = j - 10;
        a = t / 14;
        k = plane_k(t % 14, dp);
        z = zp;
    }
}

// pack (lattice -> message) or unpack (message -> lattice), T the storage's raw
// type (the lattice keeps a node's two components side by side, the message
// keeps each component's entries apart)
template <class T>
__global__ void halo_copy_kernel(Layout L, T* __restrict__ f, T* __restrict__ msg, int zc, int dc, int zp, int dp,
                                 int unpack)
{
    const int nxy = L.nx * L.ny;
    const int n = kHaloEntries * nxy;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int j = i / nxy, r = i - j * nxy;
        const int y = r / L.nx, x = r - y * L.nx;
        int a, k, z;
        entry_of(j, zc, dc, zp, dp, a, k, z);
        T* p = f + L.at(a, k, L.off(x, y, z));
        if (unpack) *p = msg[i];
        else msg[i] = *p;
    }
}

// both directions of the face between slab A (below) and slab B (above),
// lattice to lattice: A's "up" message into B, B's "down" message into A
template <class T>
__global__ void halo_exchange_kernel(Layout LA, T* __restrict__ fa, Layout LB, T* __restrict__ fb)
{
    const int nxy = LA.nx * LA.ny;
    const int n = kHaloEntries * nxy;
    const int za = LA.nz;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 2 * n; i += gridDim.x * blockDim.x) {
        const int up = i < n;
        const int e = up ? i : i - n;
        const int j = e / nxy, r = e - j * nxy;
        const int y = r / LA.nx, x = r - y * LA.nx;
        int a, k, z_src, z_dst;
        if (up) {  // A packs its top face, B unpacks at its bottom face
            entry_of(j, za - 1, +1, za - 2, +1, a, k, z_src);
            entry_of(j, 1, +1, 0, +1, a, k, z_dst);
            fb[LB.at(a, k, LB.off(x, y, z_dst))] = fa[LA.at(a, k, LA.off(x, y, z_src))];
        } else {  // B packs its bottom face, A unpacks at its top face
            entry_of(j, 0, -1, 1, -1, a, k, z_src);
            entry_of(j, za - 2, -1, za - 1, -1, a, k, z_dst);
            fa[LA.at(a, k, LA.off(x, y, z_dst))] = fb[LB.at(a, k, LB.off(x, y, z_src))];
        }
    }
}

static int halo_grid(long long n)
{
    const long long b = (n + 255) / 256;
    return (int)(b < 1 ? 1 : (b > 8192 ? 8192 : b));
}

cudaError_t launch_halo_copy(const Layout& L, void* f, size_t elem, void* msg, int face, int unpack, cudaStream_t st)
{
    // face 0 (below): pack from planes 0 (crossing down) and 1; unpack into 1 (crossing up) and 0
    // face 1 (above): pack from planes nz-1 (crossing up) and nz-2; unpack into nz-2 (crossing down) and nz-1
    int zc, dc, zp, dp;
    if (face == 0) {
        zc = unpack ? 1 : 0;
        zp = unpack ? 0 : 1;
        dc = dp = unpack ? +1 : -1;
    } else {
        zc = unpack ? L.nz - 2 : L.nz - 1;
        zp = unpack ? L.nz - 1 : L.nz - 2;
        dc = dp = unpack ? -1 : +1;
    }
    const long long n = (long long)kHaloEntries * L.nx * L.ny;
    if (elem == 4)
        halo_copy_kernel<uint32_t><<<halo_grid(n), 256, 0, st>>>(L, (uint32_t*)f, (uint32_t*)msg, zc, dc, zp, dp, unpack);
    else
        halo_copy_kernel<uint16_t><<<halo_grid(n), 256, 0, st>>>(L, (uint16_t*)f, (uint16_t*)msg, zc, dc, zp, dp, unpack);
    return cudaGetLastError();
}

cudaError_t launch_halo_exchange(const Layout& LA, void* fa, const Layout& LB, void* fb, size_t elem, cudaStream_t st)
{
    const long long n = 2LL * kHaloEntries * LA.nx * LA.ny;
    if (elem == 4)
        halo_exchange_kernel<uint32_t><<<halo_grid(n), 256, 0, st>>>(LA, (uint32_t*)fa, LB, (uint32_t*)fb);
    else
        halo_exchange_kernel<uint16_t><<<halo_grid(n), 256, 0, st>>>(LA, (uint16_t*)fa, LB, (uint16_t*)fb);
    return cudaGetLastError();
}

}  // namespace lbsc
