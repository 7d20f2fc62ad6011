// ep_kernels.cuh -- all sm_103a kernels of the voxel electrophysiology step.
#pragma once

#include "ep_common.cuh"
#include "ep_stencil.cuh"
#include "ep_aux.cuh"
