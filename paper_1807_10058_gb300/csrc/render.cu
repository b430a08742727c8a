// Headless rendering of voxel data as lattice cells (Sec. 5, Fig. 4): every
// data point of an n^3 volume is drawn as the cell that fills space around
// its lattice point, a cube on the cubic lattice (Fig. 4a) or a rhombic
// dodecahedron on the FCC lattice (Fig. 4b), with the data value as opacity
// (0 invisible, 1 opaque).  No graphics API: an orthographic emission-
// absorption ray marcher writes a grey-level image to device memory.
//
// Geometry.  Cubic: voxel (i, l, q) sits at (i, l, q); its cell is the unit
// cube around it, found by rounding every coordinate.  FCC: the lattice D3 =
// {z in Z^3 : z1 + z2 + z3 even}, voxel (i, l, q) at z = (i + q, i + l, l + q)
// (basis (1,1,0), (0,1,1), (1,0,1)); its cell is the Voronoi cell of z, the
// rhombic dodecahedron |x_a - z_a| + |x_b - z_b| <= 1 (a != b), found as the
// nearest point of D3: round every coordinate, and if the rounded coordinates
// have an odd sum, round the coordinate with the largest rounding error the
// other way (the decoding rule of Conway and Sloane for D_n).
//
// Camera: looking at the centre of the volume's bounding box from the
// direction (cos e cos a, cos e sin a, sin e) (a = azimuth, e = elevation);
// the image spans the box's bounding sphere; samples every `step` along each
// ray; a sample in a cell of value v (clamped to [0, 1]) has opacity
// 1 - exp(-kappa v step) and emits v; front-to-back compositing, stopping at
// opacity 0.999.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "fcc_dct.h"

namespace fcc {
namespace {

struct Camera {
    float3 o, right, up, dir;   // image-plane centre, half-extent axes (scaled), view direction
    float t1;                   // ray length
};

__global__ void render_kernel(const float* __restrict__ vol, int n, int cells, Camera cam, float kappa, float step,
                              int width, int height, float* __restrict__ image) {
    const int px = blockIdx.x * blockDim.x + threadIdx.x, py = blockIdx.y * blockDim.y + threadIdx.y;
    if (px >= width || py >= height) return;
    const float sx = (2.f * (px + 0.5f) / width - 1.f), sy = (1.f - 2.f * (py + 0.5f) / height);
    const float3 o = make_float3(cam.o.x + sx * cam.right.x + sy * cam.up.x, cam.o.y + sx * cam.right.y + sy * cam.up.y,
                                 cam.o.z + sx * cam.right.z + sy * cam.up.z);
    float C = 0.f, A = 0.f;
    const int nsteps = (int)(cam.t1 / step);
    // clip the ray to the occupied region (samples outside it hit no cell):
    // in voxel coordinates u = (i, l, q) -- the lattice coordinates x
    // themselves for cubes, u = B^{-1} x for the FCC lattice -- every sample
    // that decodes to a voxel of the volume lies in lo <= u_a <= hi (cubes:
    // [-1/2, n - 1/2]; a rhombic dodecahedron reaches at most 3/4 from its
    // centre in each voxel coordinate, so [-3/2, n + 1/2] keeps a margin)
    float t_in = 0.f, t_out = cam.t1;
    {
        const float lo = cells == FCC_CELL_CUBE ? -0.5f : -1.5f;
        const float hi = cells == FCC_CELL_CUBE ? (float)n - 0.5f : (float)n + 0.5f;
        float uo[3], ud[3];
        if (cells == FCC_CELL_CUBE) {
            uo[0] = o.x; uo[1] = o.y; uo[2] = o.z;
            ud[0] = cam.dir.x; ud[1] = cam.dir.y; ud[2] = cam.dir.z;
        } else {   // i = (z1 + z2 - z3) / 2, l = (z2 + z3 - z1) / 2, q = (z1 + z3 - z2) / 2
            uo[0] = 0.5f * (o.x + o.y - o.z); uo[1] = 0.5f * (o.y + o.z - o.x); uo[2] = 0.5f * (o.x + o.z - o.y);
            ud[0] = 0.5f * (cam.dir.x + cam.dir.y - cam.dir.z); ud[1] = 0.5f * (cam.dir.y + cam.dir.z - cam.dir.x);
            ud[2] = 0.5f * (cam.dir.x + cam.dir.z - cam.dir.y);
        }
        for (int a = 0; a < 3; ++a) {
            if (fabsf(ud[a]) < 1e-12f) {
                if (uo[a] < lo || uo[a] > hi) t_out = -1.f;   // parallel and outside
            } else {
                const float ta = (lo - uo[a]) / ud[a], tb = (hi - uo[a]) / ud[a];
                t_in = fmaxf(t_in, fminf(ta, tb));
                t_out = fminf(t_out, fmaxf(ta, tb));
            }
        }
    }
    // sample s sits at t = (s + 1/2) step; one sample of slack on each side
    const int s0 = t_out < t_in ? nsteps : max(0, (int)floorf(t_in / step - 0.5f) - 1);
    const int s1 = t_out < t_in ? 0 : min(nsteps, (int)ceilf(t_out / step - 0.5f) + 2);
    for (int s = s0; s < s1 && A < 0.999f; ++s) {
        const float t = (s + 0.5f) * step;
        const float x[3] = {o.x + t * cam.dir.x, o.y + t * cam.dir.y, o.z + t * cam.dir.z};
        int i, l, q;
        if (cells == FCC_CELL_CUBE) {
            i = (int)rintf(x[0]);
            l = (int)rintf(x[1]);
            q = (int)rintf(x[2]);
        } else {
            float f[3];
            int worst = 0;
            float werr = -1.f;
            for (int a = 0; a < 3; ++a) {
                f[a] = rintf(x[a]);
                const float e = fabsf(x[a] - f[a]);
                if (e > werr) { werr = e; worst = a; }
            }
            if ((((int)f[0] + (int)f[1] + (int)f[2]) & 1) != 0) f[worst] += x[worst] >= f[worst] ? 1.f : -1.f;
            const int z1 = (int)f[0], z2 = (int)f[1], z3 = (int)f[2];
            i = (z1 + z2 - z3) / 2;
            l = (z2 + z3 - z1) / 2;
            q = (z1 + z3 - z2) / 2;
        }
        if (i < 0 || l < 0 || q < 0 || i >= n || l >= n || q >= n) continue;
        const float v = fminf(fmaxf(vol[((int64_t)i * n + l) * n + q], 0.f), 1.f);
        if (v <= 0.f) continue;
        const float a = 1.f - expf(-kappa * v * step);
        C += (1.f - A) * a * v;
        A += (1.f - A) * a;
    }
    image[(int64_t)py * width + px] = C;
}

}  // namespace
}  // namespace fcc

extern "C" fcc_status fcc_render_cells(const float* volume, int n, int cells, float azimuth, float elevation,
                                       float kappa, float step, int width, int height, float* image, void* stream) {
    using namespace fcc;
    if (!volume || !image || n < 1 || n > FCC_MAX_ORDER || (cells != FCC_CELL_CUBE && cells != FCC_CELL_RHOMBIC_DODECAHEDRON) ||
        width < 1 || height < 1 || width > 16384 || height > 16384 || !(kappa > 0.f) || !(step > 0.f))
        return FCC_ERR_INVALID_ARG;
    // bounding box of the cells, its centre and bounding sphere
    const float lo = cells == FCC_CELL_CUBE ? -0.5f : -1.f;
    const float hi = cells == FCC_CELL_CUBE ? (float)n - 0.5f : 2.f * (float)n - 1.f;
    const float c = 0.5f * (lo + hi), r = 0.5f * (hi - lo) * sqrtf(3.f);
    if (r / step > 1e6f) return FCC_ERR_INVALID_ARG;
    const float ca = cosf(azimuth), sa = sinf(azimuth), ce = cosf(elevation), se = sinf(elevation);
    const float3 v = make_float3(ce * ca, ce * sa, se);                  // towards the camera
    const float3 right = make_float3(-sa, ca, 0.f);
    const float3 up = make_float3(-se * ca, -se * sa, ce);               // v x right
    Camera cam;
    cam.dir = make_float3(-v.x, -v.y, -v.z);
    cam.o = make_float3(c + r * v.x, c + r * v.y, c + r * v.z);
    cam.right = make_float3(r * right.x, r * right.y, r * right.z);
    cam.up = make_float3(r * up.x, r * up.y, r * up.z);
    cam.t1 = 2.f * r;
    dim3 block(16, 16), grid((unsigned)((width + 15) / 16), (unsigned)((height + 15) / 16));
    render_kernel<<<grid, block, 0, (cudaStream_t)stream>>>(volume, n, cells, cam, kappa, step, width, height, image);
    return cudaGetLastError() == cudaSuccess ? FCC_OK : FCC_ERR_CUDA;
}
