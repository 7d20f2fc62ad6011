/*
 * ep_sdf.h -- C ABI of the geometry encoder: signed distance functions
 * evaluated on the voxel grid on the GPU (T. Simpson, "Computational Tools
 * for Cardiac Simulation", thesis, arXiv 2302.12519, Sec. "Geometry":
 * "Signed Distance Function", "Primitives", "Encoding"; Sec. "Fibre
 * Directions" for the fibre rule).
 *
 * A scene is a set of regions, each a postfix program of nodes: primitive
 * nodes push their value at the point, operator nodes pop their operands and
 * push the result.  A negative value means inside.  Two passes run on the
 * device: one thread per voxel evaluates every region at the voxel centre
 * (the last region that contains it gives its kind, its tissue flag and its
 * fibre), then one thread per grid vertex classifies the vertex from the
 * voxels incident to it.  The outputs feed ep_set_mask and ep_set_fibres.
 *
 * Arithmetic that decides inside or outside is FP32, one IEEE-rounded
 * operation at a time in a fixed order (translate; rotate row by row, left
 * to right; the primitive's formula), so a CPU that evaluates the same
 * sequence takes the same decisions.
 *
 * Conventions as in ep.h: every call returns an ep_status; host buffers are
 * copied or written before the call returns; the call synchronises the given
 * stream (NULL: the legacy default stream) and allocates device memory only
 * for its own duration.
 */
#ifndef EP_SDF_H
#define EP_SDF_H

#include <stddef.h>
#include <stdint.h>

#include "ep.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Primitives (Sec. "Primitives"), in the node's local frame
 * p = rot (x - centre), rot row-major:
 *   EP_SDF_CUBOID     a, b, c = half-extents:  max_i |p_i / r_i| - 1
 *   EP_SDF_ELLIPSOID  a, b, c = semi-axes:     |p / r| - 1
 *   EP_SDF_CYLINDER   a = radius, b = half-height, axis z:
 *                     max(|p_xy| - a, |p_z| - b)
 *   EP_SDF_CONE       a = radius at p_z = 0, b = half-height, c = slope:
 *                     max(|p_xy| - c p_z - a, |p_z| - b)
 * Operators (the set algebra of Sec. "Primitives"):
 *   EP_SDF_UNION         min(s1, s2)
 *   EP_SDF_INTERSECT     max(s1, s2)
 *   EP_SDF_SUBTRACT      max(s1, -s2)       (s1 minus s2; s2 is the top of the stack)
 *   EP_SDF_HOLLOW        |s| - a             (a shell of half-thickness a)
 *   EP_SDF_SMOOTH_UNION  min(s1, s2) - h^2 a / 4, h = max(a - |s1 - s2|, 0) / a, a > 0
 *                        (the smoothed minimum; the thesis gives no formula,
 *                        this quadratic blend is the reading) */
#define EP_SDF_CUBOID 0
#define EP_SDF_ELLIPSOID 1
#define EP_SDF_CYLINDER 2
#define EP_SDF_CONE 3
#define EP_SDF_UNION 10
#define EP_SDF_INTERSECT 11
#define EP_SDF_SUBTRACT 12
#define EP_SDF_HOLLOW 13
#define EP_SDF_SMOOTH_UNION 14

typedef struct {
    int op;
    float a, b, c;       /* primitive sizes (mm) or operator parameter */
    float centre[3];     /* mm, scene frame */
    float rot[9];        /* row-major rotation into the local frame */
} ep_sdf_node;

/* Region kinds.  MYOCARDIUM: tissue, fibre by the rule of Sec. "Fibre
 * Directions" -- the horizontal unit vector orthogonal to the position vector
 * p of the voxel centre (scene frame, origin at the heart's centre),
 * h = (-p_y, p_x, 0) / |p_xy|, turned by helix_rad about p:
 * f = cos(helix) h + sin(helix) (p / |p|) x h; zero where p is vertical.
 * FAST: tissue with fibre scale * axis (a fast-conducting fibre: with
 * scale^2 = (g sigma_L - sigma_T) / (sigma_L - sigma_T) its longitudinal
 * conductivity is g sigma_L, Eq. sigma1).  INSULATOR: not tissue (zero
 * conductivity: no current crosses it). */
#define EP_REGION_MYOCARDIUM 1
#define EP_REGION_FAST 2
#define EP_REGION_INSULATOR 3

typedef struct {
    int first, count;    /* the region's program: nodes [first, first + count) */
    int kind;
    float axis[3];       /* FAST: fibre direction (unit) */
    float scale;         /* FAST: fibre length */
} ep_sdf_region;

/* Encode a scene on an nx*ny*nz grid whose voxel (i, j, k) has its centre at
 * origin_mm + (i + 1/2, j + 1/2, k + 1/2) dx_mm (each coordinate formed as
 * origin + ((float)i + 0.5f) * dx in FP32).  Regions are applied in order.
 * Outputs (each may be NULL, x fastest):
 *   label_out     n bytes: kind of the last region containing the voxel centre, 0 if none
 *   mask_out      n bytes: 1 for MYOCARDIUM and FAST voxels, else 0
 *   fibres_out    3n floats: (fx, fy, fz) per voxel, zero off the tissue
 *   vertex_out    (nx+1)(ny+1)(nz+1) bytes, vertex (I, J, K) at I + (nx+1)(J + (ny+1)K):
 *                 1 (solid) if every voxel of the grid incident to it is tissue,
 *                 0 (fluid) if none is, 2 (surface) otherwise (Sec. "Encoding")
 *   n_tissue_out  number of tissue voxels
 * EP_EINVAL for an invalid program (unknown op, an operator without
 * operands, a region that does not leave exactly one value, more than 32
 * values on the stack, a non-positive size where the formula divides by it),
 * a region range outside the nodes, an unknown kind, or a non-positive grid
 * or spacing; EP_ECUDA / EP_ENOMEM on device errors. */
ep_status ep_sdf_encode(const ep_sdf_node *nodes, int n_nodes, const ep_sdf_region *regions, int n_regions,
                        int nx, int ny, int nz, float dx_mm, const float origin_mm[3], double helix_rad,
                        uint8_t *label_out, uint8_t *mask_out, float *fibres_out, uint8_t *vertex_out,
                        long long *n_tissue_out, void *cuda_stream);

/* The same passes into device memory the caller owns, queued on
 * cuda_stream without synchronising (the node and region tables are copied
 * from host memory on that stream first).  d_nodes, d_regions: room for
 * n_nodes nodes and n_regions regions; d_mask: n bytes; d_n_tissue: one
 * unsigned 64-bit counter (set to the tissue count); d_label (n bytes),
 * d_fibres (3n floats) and d_vertex ((nx+1)(ny+1)(nz+1) bytes) may be NULL.
 * The arguments are checked as in ep_sdf_encode before anything is queued. */
ep_status ep_sdf_encode_device(const ep_sdf_node *nodes, int n_nodes, const ep_sdf_region *regions, int n_regions,
                               int nx, int ny, int nz, float dx_mm, const float origin_mm[3], double helix_rad,
                               ep_sdf_node *d_nodes, ep_sdf_region *d_regions, uint8_t *d_label, uint8_t *d_mask,
                               float *d_fibres, uint8_t *d_vertex, unsigned long long *d_n_tissue,
                               void *cuda_stream);

/* Message of the last failed ep_sdf_encode(_device) call of this thread. */
const char *ep_sdf_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
