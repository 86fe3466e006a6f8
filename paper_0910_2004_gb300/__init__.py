"""GB300 (sm_103a) coarsening, projection and cut/gain evaluation for the
multilevel graph partitioner of "Engineering a Scalable High Quality Graph
Partitioner" (Holtgrewe, Sanders, Schulz).

The computation lives in the CUDA library built from csrc/ (C ABI:
include/kp.h).  Submodules: `binding` (thin Python binding of the C ABI),
`build` (nvcc build of the library), `inputs` (seeded synthetic inputs).
"""
