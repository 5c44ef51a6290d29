"""GB300-native Voronoi point-inclusion test for convex polygons (arXiv 2007.15385)."""
