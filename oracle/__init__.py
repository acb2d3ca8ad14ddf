"""Independent CPU oracle for the hybrid demagnetization-field method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import, call,
link or execute anything in this package.  It shares no code with the CUDA
library (``paper_1910_07054_gb300``) and neither imports the other.

Contents:
  newell.c / newell_impl.h  generalized Newell tensor (Sec. 2): exact formula in
                            double and _Float128, far-field quadrature reading
  newell.py                 ctypes wrapper of that library
  demag.py                  direct real-space sum (Eq. Hi_discrete), the hybrid
                            2D-FFT method (Eq. FFT_v2) and the 3D-FFT method
                            (Eq. FFT_3D), all in float64 with numpy
"""
