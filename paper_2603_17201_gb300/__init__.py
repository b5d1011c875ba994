"""GB300-native Sim(3) essential-graph optimiser (the pose-graph step of
FastLoop's loop correction, Sec. III-B and IV-F), hand-written CUDA for sm_103a
behind a C ABI (``include/pgo.h``).

The CUDA library is loaded lazily on first use; ``synthetic`` (the seeded
input generators) imports without it.
"""
__version__ = "0.1.0"


def __getattr__(name):
    if name in ("PoseGraph", "evaluate_cost", "default_options", "PGOError", "solve_pose_graph", "PoseGraphBatch",
                "propagate_correction", "correct_points", "Frames", "match_params"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
