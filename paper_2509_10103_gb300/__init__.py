"""GB300-native forward/adjoint pipe-flow solver for nonlinear optimal perturbations.

The compute path lives in the CUDA shared library built from ``csrc/``; this
package only marshals arguments to its C ABI (``_lib``) and provides seeded
synthetic inputs (``synth``).
"""
