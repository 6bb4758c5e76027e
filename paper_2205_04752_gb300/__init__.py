"""GB300 (sm_103a) H-matrix library for the collocation Lame single-layer
operator: cluster tree and partition (host C++), near-field quadrature,
batched ACA and H-matrix-vector products (hand-written CUDA) behind the C ABI
of ``include/hmat.h``.

The binding is imported lazily so that ``paper_2205_04752_gb300.inputs``
(seeded synthetic meshes) can be used without the CUDA library.
"""

__all__ = ["build_cluster_tree", "aca_assemble", "hmatvec", "hmatvec_host", "solve", "HMatrix",
           "ClusterTree", "PointTree", "build_point_tree", "eval_points", "amvm", "VertexTree",
           "build_vertex_tree", "double_layer_matvec", "FP64", "FP32", "BF16", "FP16", "I16"]


def __getattr__(name):
    if name in __all__ or name == "HMError":
        import importlib
        return getattr(importlib.import_module(__name__ + ".binding"), name)
    raise AttributeError(name)
