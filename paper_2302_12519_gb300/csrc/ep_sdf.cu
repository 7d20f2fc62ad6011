// ep_sdf.cu -- geometry encoder: signed distance functions evaluated on the
// voxel grid (Sec. "Geometry": "Signed Distance Function", "Primitives",
// "Encoding"; Sec. "Fibre Directions").  Two passes, as the thesis encodes
// its meshes: one thread per voxel evaluates the scene at the voxel centre,
// one thread per vertex classifies the vertex from its incident voxels.
//
// Inside/outside decisions use FP32 with every operation an explicit
// round-to-nearest intrinsic, so no multiply-add is contracted and the result
// is the same on any IEEE machine that evaluates the same sequence.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "ep_sdf.h"

namespace {

constexpr int kStack = 32;
constexpr int kMaxNodes = 4096;
constexpr int kMaxRegions = 64;

thread_local std::string g_err;

ep_status sdf_fail(ep_status st, const std::string &m)
{
    g_err = m;
    return st;
}

__device__ __forceinline__ float sub_rn(float a, float b) { return __fadd_rn(a, -b); }

// Primitive value at scene point x (Sec. "Primitives").
__device__ float sdf_prim(const ep_sdf_node &nd, float x0, float x1, float x2)
{
    const float d0 = sub_rn(x0, nd.centre[0]), d1 = sub_rn(x1, nd.centre[1]), d2 = sub_rn(x2, nd.centre[2]);
    float p[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float t0 = __fmul_rn(nd.rot[3 * i], d0);
        const float t1 = __fmul_rn(nd.rot[3 * i + 1], d1);
        const float t2 = __fmul_rn(nd.rot[3 * i + 2], d2);
        p[i] = __fadd_rn(__fadd_rn(t0, t1), t2);
    }
    switch (nd.op) {
    case EP_SDF_CUBOID: {
        const float q0 = fabsf(__fdiv_rn(p[0], nd.a)), q1 = fabsf(__fdiv_rn(p[1], nd.b)),
                    q2 = fabsf(__fdiv_rn(p[2], nd.c));
        return fmaxf(sub_rn(q0, 1.0f), fmaxf(sub_rn(q1, 1.0f), sub_rn(q2, 1.0f)));
    }
    case EP_SDF_ELLIPSOID: {
        const float q0 = __fdiv_rn(p[0], nd.a), q1 = __fdiv_rn(p[1], nd.b), q2 = __fdiv_rn(p[2], nd.c);
        const float r = __fadd_rn(__fadd_rn(__fmul_rn(q0, q0), __fmul_rn(q1, q1)), __fmul_rn(q2, q2));
        return sub_rn(__fsqrt_rn(r), 1.0f);
    }
    case EP_SDF_CYLINDER: {
        const float rxy = __fsqrt_rn(__fadd_rn(__fmul_rn(p[0], p[0]), __fmul_rn(p[1], p[1])));
        return fmaxf(sub_rn(rxy, nd.a), sub_rn(fabsf(p[2]), nd.b));
    }
    default: {   // EP_SDF_CONE
        const float rxy = __fsqrt_rn(__fadd_rn(__fmul_rn(p[0], p[0]), __fmul_rn(p[1], p[1])));
        return fmaxf(sub_rn(sub_rn(rxy, __fmul_rn(nd.c, p[2])), nd.a), sub_rn(fabsf(p[2]), nd.b));
    }
    }
}

// One region's program at x; the program was validated on the host.
__device__ float sdf_eval(const ep_sdf_node *nodes, int first, int count, float x0, float x1, float x2)
{
    float st[kStack];
    int sp = 0;
    for (int i = first; i < first + count; ++i) {
        const ep_sdf_node &nd = nodes[i];
        if (nd.op < EP_SDF_UNION) {
            st[sp++] = sdf_prim(nd, x0, x1, x2);
        } else if (nd.op == EP_SDF_HOLLOW) {
            st[sp - 1] = sub_rn(fabsf(st[sp - 1]), nd.a);
        } else {
            const float b = st[--sp], a = st[--sp];
            float r;
            if (nd.op == EP_SDF_UNION) r = fminf(a, b);
            else if (nd.op == EP_SDF_INTERSECT) r = fmaxf(a, b);
            else if (nd.op == EP_SDF_SUBTRACT) r = fmaxf(a, -b);
            else {   // smoothed minimum: min(a, b) - h^2 k / 4
                const float k = nd.a;
                const float h = __fdiv_rn(fmaxf(sub_rn(k, fabsf(sub_rn(a, b))), 0.0f), k);
                r = sub_rn(fminf(a, b), __fmul_rn(__fmul_rn(__fmul_rn(h, h), k), 0.25f));
            }
            st[sp++] = r;
        }
    }
    return st[0];
}

// Volume pass: kind, tissue flag and fibre of every voxel.
__global__ void k_sdf_volume(const ep_sdf_node *nodes, const ep_sdf_region *regions, int n_regions, int nx, int ny,
                             int nz, float dx, float o0, float o1, float o2, float ca, float sa, uint8_t *label,
                             uint8_t *mask, float *fib, unsigned long long *n_tissue)
{
    const long long n = (long long)nx * ny * nz;
    unsigned long long cnt = 0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q % nx), j = (int)((q / nx) % ny), k = (int)(q / ((long long)nx * ny));
        const float x0 = __fadd_rn(o0, __fmul_rn(__fadd_rn((float)i, 0.5f), dx));
        const float x1 = __fadd_rn(o1, __fmul_rn(__fadd_rn((float)j, 0.5f), dx));
        const float x2 = __fadd_rn(o2, __fmul_rn(__fadd_rn((float)k, 0.5f), dx));
        int last = -1;
        for (int r = 0; r < n_regions; ++r)
            if (sdf_eval(nodes, regions[r].first, regions[r].count, x0, x1, x2) < 0.0f) last = r;
        const int kind = last >= 0 ? regions[last].kind : 0;
        const bool tissue = kind == EP_REGION_MYOCARDIUM || kind == EP_REGION_FAST;
        float f0 = 0.f, f1 = 0.f, f2 = 0.f;
        if (kind == EP_REGION_MYOCARDIUM) {   // helical rule of Sec. "Fibre Directions"
            const float hl = sqrtf(x0 * x0 + x1 * x1);
            if (hl > 0.f) {
                const float pl = sqrtf(x0 * x0 + x1 * x1 + x2 * x2);
                const float h0 = -x1 / hl, h1 = x0 / hl;   // h2 = 0
                const float u0 = x0 / pl, u1 = x1 / pl, u2 = x2 / pl;
                const float w0 = -u2 * h1, w1 = u2 * h0, w2 = u0 * h1 - u1 * h0;   // u x h
                f0 = ca * h0 + sa * w0;
                f1 = ca * h1 + sa * w1;
                f2 = sa * w2;
            }
        } else if (kind == EP_REGION_FAST) {
            const ep_sdf_region &rg = regions[last];
            f0 = rg.scale * rg.axis[0];
            f1 = rg.scale * rg.axis[1];
            f2 = rg.scale * rg.axis[2];
        }
        if (label) label[q] = (uint8_t)kind;
        mask[q] = tissue ? 1 : 0;
        if (fib) {
            fib[3 * q] = f0;
            fib[3 * q + 1] = f1;
            fib[3 * q + 2] = f2;
        }
        cnt += tissue ? 1 : 0;
    }
    // tissue count: warp sum, one atomic per warp
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(n_tissue, cnt);
}

// Vertex pass (Sec. "Encoding"): 1 solid, 0 fluid, 2 surface.
__global__ void k_sdf_vertex(const uint8_t *mask, int nx, int ny, int nz, uint8_t *vclass)
{
    const long long nv = (long long)(nx + 1) * (ny + 1) * (nz + 1);
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nv; v += (long long)gridDim.x * blockDim.x) {
        const int I = (int)(v % (nx + 1)), J = (int)((v / (nx + 1)) % (ny + 1)),
                  K = (int)(v / ((long long)(nx + 1) * (ny + 1)));
        int in = 0, tis = 0;
        for (int u = 0; u < 2; ++u)
            for (int t = 0; t < 2; ++t)
                for (int s = 0; s < 2; ++s) {
                    const int i = I - 1 + s, j = J - 1 + t, k = K - 1 + u;
                    if (i < 0 || j < 0 || k < 0 || i >= nx || j >= ny || k >= nz) continue;
                    ++in;
                    tis += mask[(long long)i + (long long)nx * ((long long)j + (long long)ny * k)];
                }
        vclass[v] = (uint8_t)(tis == 0 ? 0 : (tis == in ? 1 : 2));
    }
}

int grid_of(long long n, int threads)
{
    const long long g = (n + threads - 1) / threads;
    return (int)std::max<long long>(1, std::min<long long>(g, 152LL * 64));
}

// Host validation of one region's program: stack effects, operands, sizes.
bool check_program(const ep_sdf_node *nodes, int first, int count, std::string &why)
{
    int depth = 0;
    for (int i = first; i < first + count; ++i) {
        const ep_sdf_node &nd = nodes[i];
        switch (nd.op) {
        case EP_SDF_CUBOID: case EP_SDF_ELLIPSOID:
            if (!(nd.a > 0.f && nd.b > 0.f && nd.c > 0.f)) { why = "cuboid / ellipsoid sizes must be > 0"; return false; }
            ++depth;
            break;
        case EP_SDF_CYLINDER: case EP_SDF_CONE:
            if (!std::isfinite(nd.a) || !std::isfinite(nd.b) || !std::isfinite(nd.c)) { why = "non-finite size"; return false; }
            ++depth;
            break;
        case EP_SDF_HOLLOW:
            if (depth < 1 || !std::isfinite(nd.a)) { why = "hollow needs an operand and a finite thickness"; return false; }
            break;
        case EP_SDF_SMOOTH_UNION:
            if (!(nd.a > 0.f) || !std::isfinite(nd.a)) { why = "smooth union width must be > 0"; return false; }
            /* fall through */
        case EP_SDF_UNION: case EP_SDF_INTERSECT: case EP_SDF_SUBTRACT:
            if (depth < 2) { why = "an operator is missing an operand"; return false; }
            --depth;
            break;
        default:
            why = "unknown node op";
            return false;
        }
        if (depth > kStack) { why = "more than 32 values on the stack"; return false; }
        for (int c = 0; c < 3; ++c)
            if (!std::isfinite(nd.centre[c])) { why = "non-finite centre"; return false; }
        for (int c = 0; c < 9; ++c)
            if (!std::isfinite(nd.rot[c])) { why = "non-finite rotation"; return false; }
    }
    if (depth != 1) { why = "a region's program must leave exactly one value"; return false; }
    return true;
}

// Argument checks shared by both entry points.
ep_status sdf_check(const ep_sdf_node *nodes, int n_nodes, const ep_sdf_region *regions, int n_regions, int nx,
                    int ny, int nz, float dx_mm, const float origin_mm[3], double helix_rad)
{
    if (!nodes || !regions || !origin_mm) return sdf_fail(EP_EINVAL, "nodes, regions and origin must be given");
    if (n_nodes < 1 || n_nodes > kMaxNodes) return sdf_fail(EP_EINVAL, "1..4096 nodes");
    if (n_regions < 1 || n_regions > kMaxRegions) return sdf_fail(EP_EINVAL, "1..64 regions");
    if (nx < 1 || ny < 1 || nz < 1) return sdf_fail(EP_EINVAL, "grid dimensions must be >= 1");
    if ((long long)nx * ny * nz > 2147483647LL) return sdf_fail(EP_EINVAL, "grid too large");
    if (!(dx_mm > 0.f) || !std::isfinite(dx_mm)) return sdf_fail(EP_EINVAL, "dx must be > 0");
    if (!std::isfinite(helix_rad)) return sdf_fail(EP_EINVAL, "helix angle must be finite");
    for (int c = 0; c < 3; ++c)
        if (!std::isfinite(origin_mm[c])) return sdf_fail(EP_EINVAL, "origin must be finite");
    for (int r = 0; r < n_regions; ++r) {
        const ep_sdf_region &rg = regions[r];
        if (rg.first < 0 || rg.count < 1 || rg.first + rg.count > n_nodes)
            return sdf_fail(EP_EINVAL, "region program outside the nodes");
        if (rg.kind != EP_REGION_MYOCARDIUM && rg.kind != EP_REGION_FAST && rg.kind != EP_REGION_INSULATOR)
            return sdf_fail(EP_EINVAL, "unknown region kind");
        std::string why;
        if (!check_program(nodes, rg.first, rg.count, why)) return sdf_fail(EP_EINVAL, why);
    }
    return EP_OK;
}

}  // namespace

extern "C" {

const char *ep_sdf_last_error(void) { return g_err.c_str(); }

ep_status ep_sdf_encode_device(const ep_sdf_node *nodes, int n_nodes, const ep_sdf_region *regions, int n_regions,
                               int nx, int ny, int nz, float dx_mm, const float origin_mm[3], double helix_rad,
                               ep_sdf_node *d_nodes, ep_sdf_region *d_regions, uint8_t *d_label, uint8_t *d_mask,
                               float *d_fibres, uint8_t *d_vertex, unsigned long long *d_n_tissue,
                               void *cuda_stream)
{
    ep_status v = sdf_check(nodes, n_nodes, regions, n_regions, nx, ny, nz, dx_mm, origin_mm, helix_rad);
    if (v != EP_OK) return v;
    if (!d_nodes || !d_regions || !d_mask || !d_n_tissue) return sdf_fail(EP_EINVAL, "device buffers must be given");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const long long n = (long long)nx * ny * nz, nv = (long long)(nx + 1) * (ny + 1) * (nz + 1);
    cudaError_t e = cudaMemcpyAsync(d_nodes, nodes, sizeof(ep_sdf_node) * n_nodes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_regions, regions, sizeof(ep_sdf_region) * n_regions, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_n_tissue, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return sdf_fail(EP_ECUDA, std::string("copy: ") + cudaGetErrorString(e));
    k_sdf_volume<<<grid_of(n, 256), 256, 0, st>>>(d_nodes, d_regions, n_regions, nx, ny, nz, dx_mm, origin_mm[0],
                                                  origin_mm[1], origin_mm[2], (float)std::cos(helix_rad),
                                                  (float)std::sin(helix_rad), d_label, d_mask, d_fibres, d_n_tissue);
    if (d_vertex) k_sdf_vertex<<<grid_of(nv, 256), 256, 0, st>>>(d_mask, nx, ny, nz, d_vertex);
    e = cudaGetLastError();
    if (e != cudaSuccess) return sdf_fail(EP_ECUDA, std::string("encode kernels: ") + cudaGetErrorString(e));
    return EP_OK;
}

ep_status ep_sdf_encode(const ep_sdf_node *nodes, int n_nodes, const ep_sdf_region *regions, int n_regions,
                        int nx, int ny, int nz, float dx_mm, const float origin_mm[3], double helix_rad,
                        uint8_t *label_out, uint8_t *mask_out, float *fibres_out, uint8_t *vertex_out,
                        long long *n_tissue_out, void *cuda_stream)
{
    ep_status v = sdf_check(nodes, n_nodes, regions, n_regions, nx, ny, nz, dx_mm, origin_mm, helix_rad);
    if (v != EP_OK) return v;
    const long long n = (long long)nx * ny * nz;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const long long nv = (long long)(nx + 1) * (ny + 1) * (nz + 1);
    ep_sdf_node *d_nodes = nullptr;
    ep_sdf_region *d_reg = nullptr;
    uint8_t *d_label = nullptr, *d_mask = nullptr, *d_v = nullptr;
    float *d_fib = nullptr;
    unsigned long long *d_cnt = nullptr;
    ep_status ret = EP_OK;
    auto ck = [&](cudaError_t e, const char *what) {
        if (e != cudaSuccess && ret == EP_OK) {
            ret = e == cudaErrorMemoryAllocation ? EP_ENOMEM : EP_ECUDA;
            g_err = std::string(what) + ": " + cudaGetErrorString(e);
        }
        return e == cudaSuccess;
    };
    if (ck(cudaMalloc(&d_nodes, sizeof(ep_sdf_node) * n_nodes), "cudaMalloc") &&
        ck(cudaMalloc(&d_reg, sizeof(ep_sdf_region) * n_regions), "cudaMalloc") &&
        ck(cudaMalloc(&d_mask, n), "cudaMalloc") && ck(cudaMalloc(&d_cnt, sizeof(unsigned long long)), "cudaMalloc") &&
        (!label_out || ck(cudaMalloc(&d_label, n), "cudaMalloc")) &&
        (!fibres_out || ck(cudaMalloc(&d_fib, sizeof(float) * 3 * n), "cudaMalloc")) &&
        (!vertex_out || ck(cudaMalloc(&d_v, nv), "cudaMalloc"))) {
        ret = ep_sdf_encode_device(nodes, n_nodes, regions, n_regions, nx, ny, nz, dx_mm, origin_mm, helix_rad,
                                   d_nodes, d_reg, d_label, d_mask, d_fib, d_v, d_cnt, cuda_stream);
        unsigned long long cnt = 0;
        if (ret == EP_OK) {
            if (mask_out) ck(cudaMemcpyAsync(mask_out, d_mask, n, cudaMemcpyDeviceToHost, st), "copy mask");
            if (label_out) ck(cudaMemcpyAsync(label_out, d_label, n, cudaMemcpyDeviceToHost, st), "copy labels");
            if (fibres_out)
                ck(cudaMemcpyAsync(fibres_out, d_fib, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost, st), "copy fibres");
            if (vertex_out) ck(cudaMemcpyAsync(vertex_out, d_v, nv, cudaMemcpyDeviceToHost, st), "copy vertices");
            ck(cudaMemcpyAsync(&cnt, d_cnt, sizeof(cnt), cudaMemcpyDeviceToHost, st), "copy count");
        }
        ck(cudaStreamSynchronize(st), "synchronize");
        if (n_tissue_out && ret == EP_OK) *n_tissue_out = (long long)cnt;
    }
    for (void *p : {(void *)d_nodes, (void *)d_reg, (void *)d_label, (void *)d_mask, (void *)d_v, (void *)d_fib,
                    (void *)d_cnt})
        if (p) cudaFree(p);
    return ret;
}

}  // extern "C"
