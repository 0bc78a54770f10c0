"""GB300-native embedding similarity join (top-k / threshold / contrastive).

The join evaluates C = A B^T over unit-norm float32 embeddings on sm_103a
tensor cores and returns exact results (see include/sj.h).  Submodules:

* ``sj``      -- ctypes binding of libsj.so (the C ABI) and a torch-facing
                 ``SimilarityJoin`` handle;
* ``datagen`` -- seeded synthetic workloads;
* ``_build``  -- in-tree nvcc build of libsj.so.
"""

__all__ = ["sj", "datagen"]
