"""B300-native PSDF hot path (polygonal signed distance, value + gradient).

The CUDA library (``libpsdf_b300.so``, C ABI declared in ``include/psdf.h``)
does all of the arithmetic; ``psdf`` is its thin ctypes binding and
``autograd`` wraps it in ``torch.autograd.Function``.  ``scenegen`` builds
seeded synthetic inputs.
"""
