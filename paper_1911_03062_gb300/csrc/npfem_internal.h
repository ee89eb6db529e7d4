// npfem_internal.h -- kernels of the npFEM CUDA path, collected for npfem.cu.
#pragma once

#include "common.cuh"
#include "local.cuh"
#include "step_kernels.cuh"
#include "gemm_simt.cuh"
#include "gemm_tc.cuh"
#include "gemm_grouped.cuh"
#include "residual_ell.cuh"
#include "filters.cuh"
#include "contact.cuh"
#include "ibm.cuh"
