// Instantiation of the persistent N-1 kernel (fdpf_kernel.cuh) with B''
// extension rows: for generator outages (the bus whose generator trips,
// Sec. IV.A, the loss of a single component) and for grids whose PV
// generators have reactive limits (buses held at a limit turn PQ).  Tiles
// of 2, 4 and 8 scenarios.
#include "fdpf_kernel.cuh"

namespace gpcg {

template <typename VT>
cudaError_t launch_fdpf_gen(cudaStream_t st, int T, int grid, const FdpfParams& P,
                            const DevMatT<VT>& MP, const DevMatT<VT>& MQ) {
  return launch_fdpf_g<true, VT>(st, T, grid, P, MP, MQ);
}

template <typename VT>
int fdpf_blocks_gen(int T) {
  return fdpf_blocks_g<true, VT>(T);
}

template cudaError_t launch_fdpf_gen<float>(cudaStream_t, int, int, const FdpfParams&,
                                            const DevMatT<float>&, const DevMatT<float>&);
template cudaError_t launch_fdpf_gen<double>(cudaStream_t, int, int, const FdpfParams&,
                                             const DevMatT<double>&, const DevMatT<double>&);
template int fdpf_blocks_gen<float>(int);
template int fdpf_blocks_gen<double>(int);

}  // namespace gpcg
