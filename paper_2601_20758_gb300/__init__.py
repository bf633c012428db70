"""GB300-native adaptive kernel density estimation over a region of interest
(ScaleFree, arXiv 2601.20758), behind the C ABI of include/scalefree.h.

* ``paper_2601_20758_gb300._lib``   ctypes binding of libscalefree.so
* ``paper_2601_20758_gb300.synth``  seeded synthetic clouds and ROI lists
* ``paper_2601_20758_gb300.build``  in-tree nvcc build for sm_103a

The binding is imported lazily so that the input generators can be used on a
machine without the CUDA library.
"""
