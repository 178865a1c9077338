"""GB300 (sm_103a) GIGAQBX: FMM-accelerated QBX evaluation of 3D Laplace layer potentials.

The C ABI is include/qbx.h (libqbx.so, built from csrc/ by build.py); binding.py
marshals PyTorch CUDA tensors into it.
"""
from .binding import (  # noqa: F401
    LIST_NAMES,
    STAGE_NAMES,
    QBX_FP64,
    QBX_M2L_3XTF32,
    QBX_M2L_FP32,
    Lists,
    QbxError,
    Tree,
    lib,
    library_path,
    qbx_build_lists,
    qbx_build_tree,
    qbx_eval,
    qbx_eval_noalloc,
    qbx_eval_order_sweep,
    qbx_lists_cost,
    MLP_NPARAMS,
    qbx_center_features,
    qbx_order_labels,
    qbx_mlp_init,
    qbx_mlp_forward,
    qbx_mlp_loss_grad,
    qbx_mlp_train,
    qbx_orders_from_mlp,
    Graph,
    qbx_build_forest,
    qbx_graph_create,
    qbx_lists_set_tiles,
    qbx_lists_set_wait,
    qbx_peak_flops,
    QBX_PEAK_FP64,
    QBX_PEAK_FP32,
)
