"""GB300-native forward/adjoint pipe-flow solver for nonlinear optimal perturbations.

The compute path lives in the CUDA shared library built from ``csrc/``
(``build``).  The Python modules around it run no arithmetic of the method:
``_lib`` marshals arguments to the C ABI (contexts and batches), ``autograd``
wraps the checkpointed sweep as a ``torch.autograd.Function``, ``serving``
admits and schedules gradient requests, ``diagnostics`` combines the
library's per-mode energies, and ``synth`` makes seeded synthetic inputs.
"""
