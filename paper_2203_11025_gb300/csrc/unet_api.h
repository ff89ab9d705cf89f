// Internal bridge between the solver driver and the U-Net preconditioners.
#pragma once
#include <cuda_runtime.h>

#include "../../include/unet.h"

struct helm_ctx;

// z = U-Net-based preconditioner applied to v (Alg. 2 for HELM_PREC_JU,
// Eq. 3.4 for HELM_PREC_VU); real_bytes = sizeof(real type) of v and z.
int unet_precond_impl(helm_ctx* c, void* net, int kind, const void* v, void* z, int nrhs, int real_bytes,
                      const int* gate, cudaStream_t s);
// Release U-Net workspace attached to a solver handle.
void unet_release_ctx(helm_ctx* c);
// Allocate the network's workspace for nrhs right-hand sides on c's grid (before graph capture).
int unet_prepare_impl(helm_ctx* c, void* net, int nrhs);
// Identity of the device buffers a captured cycle with this network references: {network
// id, workspace generation, encoder id, encoder workspace generation}; ids are never
// reused, generations change whenever a workspace is reallocated.
void unet_graph_ids(void* net, unsigned long long ids[4]);
// The configuration a network was created with.
void unet_cfg_of(unet_t net, unet_cfg* cfg);
