"""GB300-native NURBS-Diff hot path: batched rational B-spline curve and surface
evaluation and its backward pass, behind the C-ABI library ``libnurbs``."""
