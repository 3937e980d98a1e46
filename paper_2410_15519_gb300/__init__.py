"""GB300 (sm_103a) CTD solver for the Allen-Cahn equation (Lu, Yuan & Guo, arXiv 2410.15519).

``ctd``   ctypes binding of the C ABI in ``include/ctd.h`` (library ``libctd.so``)
``build`` in-tree nvcc build of ``libctd.so``
Importing the package loads nothing; the library is loaded on first use.
"""
