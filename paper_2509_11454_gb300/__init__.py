"""GB300-native PercIS: importance-sampling percolation centrality.

The compute path is libpercis.so (hand-written sm_103a CUDA kernels behind
the C ABI in include/percis.h); `binding` marshals arguments for it and
`synth` builds seeded synthetic inputs.  Import `binding` explicitly; this
package import itself loads nothing.
"""
__all__ = ["binding", "synth", "build_lib"]
