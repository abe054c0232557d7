// coupled_kernels.cu -- coupled rows (Alg. 2); filled in below the segmented path.
#include "dev_common.cuh"
#include "kernels.h"

namespace pgdto {

struct CoupledWork {
    GridCtrl ctrl;
    DeviceInfo info;
};

size_t coupled_work_bytes() { return sizeof(CoupledWork); }
size_t coupled_work_ctrl_bytes() { return sizeof(GridCtrl); }
DeviceInfo* coupled_work_info(CoupledWork* ws) { return &ws->info; }

cudaError_t launch_coupled(const CoupledArgs&, int, cudaStream_t) { return cudaErrorNotSupported; }
int max_blocks_coupled(int) { return 1; }

}  // namespace pgdto
