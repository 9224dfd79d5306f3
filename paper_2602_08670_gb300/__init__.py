"""GB300-native finite-volume solver for 2D shallow water and 2D Euler with a
learned-stencil variant.  The numerical work runs in the CUDA library
``_build/libfv.so`` (sources in ``csrc/``, C ABI in ``include/fv.h``);
``fv`` is its Python binding and ``workloads`` builds seeded inputs."""
