"""Seeded synthetic pangenome variation graphs and initial layouts.

This package only builds inputs. It holds none of the layout method's
arithmetic, so the CPU oracle and the CUDA library can both be fed from it.
"""
from .pangenome import CONFIGS, Graph, make_graph, make_linear_path, make_custom
from .batch import BATCH_CONFIGS, BatchArrays, batch_shapes, concat, make_batch

__all__ = ["CONFIGS", "Graph", "make_graph", "make_linear_path", "make_custom",
           "BATCH_CONFIGS", "BatchArrays", "batch_shapes", "concat", "make_batch"]
